"""GB300 (sm_103a) RKHS point-cloud registration (arXiv:2012.03683).

A thin ctypes binding over ``libcvo.so`` (include/cvo.h).  It only marshals
arguments: every step of the computation runs in the library's CUDA kernels.
PyTorch supplies device memory and the current CUDA stream.  There is no CPU
fallback: without the built library (``python -m
paper_2012_03683_gb300.build``) every call raises.

Functions named like the C entry points (``cvo_create``, ``cvo_inner_product``,
``cvo_gradient``, ``cvo_metric``, ``cvo_evaluate``, ``cvo_register_pair``,
``cvo_register_batch``, ...) take the same arguments in Python form; the
``CVO`` class wraps a handle.

Clouds are (N, 3) float32 arrays: torch CUDA tensors are passed as device
pointers, numpy arrays and CPU tensors as host pointers (the library copies
them).  Features are (N, D) float32 or bfloat16 (torch.bfloat16) arrays, the
blocks concatenated in the order given.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

__all__ = ["CVO", "cvo_create", "cvo_destroy", "cvo_set_params", "cvo_inner_product", "cvo_gradient", "cvo_metric",
           "cvo_evaluate", "cvo_backward", "cvo_metric_backward", "cvo_cosine", "CVOInnerProduct", "CVOMetric",
           "inner_product_fn", "metric_fn",
           "cvo_register_pair", "cvo_register_batch", "cvo_register_sequence", "cvo_get_trace", "cvo_set_timing",
           "cvo_autotune", "cvo_autotune_batch", "cvo_get_tuning", "cvo_apply_tuning", "cvo_set_loop",
           "cvo_sweep_time", "cvo_last_error", "cvo_version", "cvo_kernel_launches", "load_library", "Status",
           "CvoError", "cvo_shard_begin", "cvo_shard_sweep", "cvo_shard_step", "cvo_shard_end", "shard_rows",
           "register_sharded", "SHARD_STATS", "cvo_cosine_dell", "cosine_fn", "cvo_inject_barrier_stall"]

MAX_BLOCKS = 4
TRACE_STRIDE = 22
SHARD_STATS = 45


class Status:
    OK = 0
    NOT_CONVERGED = 1
    ERR_INVALID_ARG = -1
    ERR_CUDA = -2
    ERR_OOM = -3
    ERR_TIMEOUT = -4


class CvoError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"cvo status {status}: {msg}")
        self.status = status


class FeatBlock(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("kind", ctypes.c_int), ("scale", ctypes.c_double), ("sigma", ctypes.c_double)]


class Cloud(ctypes.Structure):
    _fields_ = [("xyz", ctypes.c_void_p), ("n", ctypes.c_int), ("feat", ctypes.c_void_p), ("feat_dtype", ctypes.c_int),
                ("on_device", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("ell", ctypes.c_double), ("ell_min", ctypes.c_double), ("sigma", ctypes.c_double),
                ("cutoff_mult", ctypes.c_double), ("n_blocks", ctypes.c_int), ("blocks", FeatBlock * MAX_BLOCKS),
                ("max_iters", ctypes.c_int), ("anneal", ctypes.c_int), ("decay", ctypes.c_double),
                ("indicator_tol", ctypes.c_double), ("step_tol_rot", ctypes.c_double),
                ("step_tol_trans", ctypes.c_double), ("max_step_rot", ctypes.c_double),
                ("max_step_trans", ctypes.c_double), ("feat_cutoff_mult", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("status", ctypes.c_int), ("ell_final", ctypes.c_double),
                ("F", ctypes.c_double), ("i_theta", ctypes.c_double), ("last_step_rot", ctypes.c_double),
                ("last_step_trans", ctypes.c_double), ("pairs", ctypes.c_longlong),
                ("candidates", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tuning(ctypes.Structure):
    _fields_ = [("cell_factor", ctypes.c_double), ("super_delta", ctypes.c_int), ("chunk_len", ctypes.c_int),
                ("measured_ms", ctypes.c_double), ("query_lanes", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Eval(ctypes.Structure):
    _fields_ = [("F", ctypes.c_double), ("grad", ctypes.c_double * 6), ("hess", ctypes.c_double * 36),
                ("i_theta", ctypes.c_double), ("pairs", ctypes.c_longlong), ("candidates", ctypes.c_longlong)]


class Throughput(ctypes.Structure):
    _fields_ = [("ffma_flops", ctypes.c_double), ("ex2_per_s", ctypes.c_double), ("ms_ffma", ctypes.c_double),
                ("ms_ex2", ctypes.c_double), ("sms", ctypes.c_int)]


_lib = None


def load_library(build_if_missing: bool = True):
    """Loads libcvo.so (building it first when missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not _build.up_to_date():
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"libcvo.so is not built ({path}); run python -m paper_2012_03683_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    lib.cvo_create.argtypes = [P(Params), vp, P(vp)]
    lib.cvo_destroy.argtypes = [vp]
    lib.cvo_set_params.argtypes = [vp, P(Params)]
    for name in ("cvo_inner_product", "cvo_metric"):
        getattr(lib, name).argtypes = [vp, P(Cloud), P(Cloud), vp, P(ctypes.c_double)]
    lib.cvo_gradient.argtypes = [vp, P(Cloud), P(Cloud), vp, vp, P(ctypes.c_double)]
    lib.cvo_evaluate.argtypes = [vp, P(Cloud), P(Cloud), vp, P(Eval)]
    lib.cvo_cosine.argtypes = [vp, P(Cloud), P(Cloud), vp, vp, P(ctypes.c_double), vp]
    lib.cvo_cosine_dell.argtypes = [vp, P(Cloud), P(Cloud), vp, P(ctypes.c_double), P(ctypes.c_double)]
    for name in ("cvo_backward", "cvo_metric_backward"):
        getattr(lib, name).argtypes = [vp, P(Cloud), P(Cloud), vp, ctypes.c_double, vp, vp, vp, vp,
                                       P(ctypes.c_double), ctypes.c_int]
    lib.cvo_register_pair.argtypes = [vp, P(Cloud), P(Cloud), vp, vp, P(Info)]
    lib.cvo_register_batch.argtypes = [vp, ctypes.c_int, P(Cloud), P(Cloud), vp, vp, P(Info)]
    lib.cvo_get_trace.argtypes = [vp, vp, ctypes.c_int]
    lib.cvo_register_sequence.argtypes = [vp, ctypes.c_int, P(Cloud), ctypes.c_double, vp, vp, vp, P(Info)]
    lib.cvo_set_timing.argtypes = [vp, ctypes.c_int]
    lib.cvo_set_tuning.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    lib.cvo_set_tuning.restype = ctypes.c_int
    lib.cvo_sweep_time.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_int)]
    lib.cvo_autotune.argtypes = [vp, P(Cloud), P(Cloud), vp, P(Tuning)]
    lib.cvo_autotune_batch.argtypes = [vp, ctypes.c_int, P(Cloud), P(Cloud), vp, P(Tuning)]
    lib.cvo_set_loop.argtypes = [vp, ctypes.c_int]
    lib.cvo_inject_barrier_stall.argtypes = [vp, ctypes.c_int, ctypes.c_uint]
    lib.cvo_shard_begin.argtypes = [vp, P(Cloud), P(Cloud), ctypes.c_longlong, vp]
    lib.cvo_shard_sweep.argtypes = [vp, vp]
    lib.cvo_shard_step.argtypes = [vp, vp, P(ctypes.c_int)]
    lib.cvo_shard_end.argtypes = [vp, vp, P(Info)]
    lib.cvo_get_tuning.argtypes = [vp, P(Tuning)]
    lib.cvo_apply_tuning.argtypes = [vp, P(Tuning)]
    for name in ("cvo_create", "cvo_destroy", "cvo_set_params", "cvo_inner_product", "cvo_metric", "cvo_gradient",
                 "cvo_evaluate", "cvo_backward", "cvo_metric_backward", "cvo_cosine", "cvo_register_pair",
                 "cvo_register_sequence",
                 "cvo_register_batch", "cvo_get_trace", "cvo_set_timing", "cvo_sweep_time", "cvo_autotune",
                 "cvo_autotune_batch",
                 "cvo_get_tuning", "cvo_apply_tuning", "cvo_set_loop", "cvo_shard_begin", "cvo_shard_sweep",
                 "cvo_cosine_dell", "cvo_inject_barrier_stall",
                 "cvo_shard_step", "cvo_shard_end"):
        getattr(lib, name).restype = ctypes.c_int
    lib.cvo_last_error.restype = ctypes.c_char_p
    lib.cvo_last_error.argtypes = []
    lib.cvo_version.restype = ctypes.c_char_p
    lib.cvo_version.argtypes = []
    lib.cvo_measure_throughput.restype = ctypes.c_int
    lib.cvo_measure_throughput.argtypes = [vp, P(Throughput)]
    lib.cvo_kernel_launches.restype = ctypes.c_longlong
    lib.cvo_kernel_launches.argtypes = []
    _lib = lib
    return lib


def cvo_measure_throughput(stream=None) -> dict:
    """Measured FP32 FMA and ex2 rates of the current device
    (cvo_measure_throughput): ffma_flops (FLOP/s), ex2_per_s, the best
    launch times (ms) and the SM count."""
    t = Throughput()
    s = _current_stream() if stream is None else ctypes.c_void_p(int(stream))
    _check(load_library().cvo_measure_throughput(s, ctypes.byref(t)))
    return {"ffma_flops": t.ffma_flops, "ex2_per_s": t.ex2_per_s, "ms_ffma": t.ms_ffma, "ms_ex2": t.ms_ex2,
            "sms": t.sms}


def cvo_kernel_launches() -> int:
    return int(load_library().cvo_kernel_launches())


def cvo_last_error() -> str:
    return load_library().cvo_last_error().decode()


def cvo_version() -> str:
    return load_library().cvo_version().decode()


def _check(rc):
    if rc < 0:
        raise CvoError(rc, cvo_last_error())
    return rc


# ---- argument marshalling ----------------------------------------------------

def _torch():
    try:
        import torch
        return torch
    except Exception:  # pragma: no cover
        return None


def _current_stream():
    torch = _torch()
    if torch is not None and torch.cuda.is_available() and torch.cuda.is_initialized():
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(0)


def make_params(blocks=(), ell=0.1, ell_min=None, sigma=1.0, cutoff_mult=3.0, max_iters=100, anneal=False, decay=0.98,
                indicator_tol=1e-3, step_tol_rot=1e-5, step_tol_trans=1e-5, max_step_rot=0.1,
                max_step_trans=0.0, feat_cutoff_mult=0.0) -> Params:
    """blocks: sequence of (kind, dim, scale, sigma), kind "se" (Eq. newscalar) or "dot" (Eq. scalar).
    feat_cutoff_mult > 0 also drops pairs whose "se" features lie further apart than
    feat_cutoff_mult * scale in any block (the feature-space sparsity of Sec. III-B)."""
    p = Params()
    p.ell = float(ell)
    p.ell_min = float(ell if ell_min is None else ell_min)
    p.sigma = float(sigma)
    p.cutoff_mult = float(cutoff_mult)
    blocks = list(blocks)
    if len(blocks) > MAX_BLOCKS:
        raise ValueError("at most 4 feature blocks")
    p.n_blocks = len(blocks)
    for b, (kind, dim, scale, sig) in enumerate(blocks):
        p.blocks[b].dim = int(dim)
        p.blocks[b].kind = {"se": 0, "dot": 1}[kind]
        p.blocks[b].scale = float(scale)
        p.blocks[b].sigma = float(sig)
    p.max_iters = int(max_iters)
    p.anneal = int(bool(anneal))
    p.decay = float(decay)
    p.indicator_tol = float(indicator_tol)
    p.step_tol_rot = float(step_tol_rot)
    p.step_tol_trans = float(step_tol_trans)
    p.max_step_rot = float(max_step_rot)
    p.max_step_trans = float(max_step_trans)
    p.feat_cutoff_mult = float(feat_cutoff_mult)
    return p


def _as_cloud(xyz, feat, keep):
    """Builds a Cloud from numpy arrays or torch tensors; keep holds references."""
    torch = _torch()
    if torch is not None and isinstance(xyz, torch.Tensor):
        # (a batch marshals 2 clouds per pair: no tensor is copied or
        # detached unless it has to be)
        t = xyz.detach() if xyz.requires_grad else xyz
        if t.dtype != torch.float32 or t.dim() != 2 or t.shape[1] != 3:
            raise ValueError("xyz must be an (N, 3) float32 tensor")
        if not t.is_contiguous():
            t = t.contiguous()
        keep.append(t)
        n = t.shape[0]
        cuda = t.is_cuda
        fptr, fdt = None, 0
        if feat is not None:
            f = feat.detach() if feat.requires_grad else feat
            if f.is_cuda != cuda:
                raise ValueError("xyz and features must live on the same device")
            if f.dtype == torch.bfloat16:
                fdt = 1
            elif f.dtype != torch.float32:
                raise ValueError("features must be float32 or bfloat16")
            if not f.is_contiguous():
                f = f.contiguous()
            keep.append(f)
            fptr = f.data_ptr() if f.numel() else None
        return Cloud(t.data_ptr() if n else None, n, fptr, fdt, 1 if cuda else 0)
    c = Cloud()
    a = np.ascontiguousarray(np.asarray(xyz, dtype=np.float32).reshape(-1, 3))
    keep.append(a)
    c.xyz = a.ctypes.data if a.size else None
    c.n = a.shape[0]
    c.on_device = 0
    if feat is not None:
        f = np.asarray(feat)
        if f.dtype == np.uint16:  # bfloat16 bit patterns
            c.feat_dtype = 1
        else:
            f = f.astype(np.float32, copy=False)
            c.feat_dtype = 0
        f = np.ascontiguousarray(f)
        keep.append(f)
        c.feat = f.ctypes.data if f.size else None
    return c


def _pose(T):
    a = np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(4, 4))
    return a


# ---- the C entry points --------------------------------------------------------

def cvo_create(params: Params, stream=None):
    lib = load_library()
    h = ctypes.c_void_p()
    s = _current_stream() if stream is None else ctypes.c_void_p(int(stream))
    _check(lib.cvo_create(ctypes.byref(params), s, ctypes.byref(h)))
    return h


def cvo_destroy(h):
    return _check(load_library().cvo_destroy(h))


def cvo_set_params(h, params: Params):
    return _check(load_library().cvo_set_params(h, ctypes.byref(params)))


def _clouds(X, Z, FX, FZ):
    keep = []
    return _as_cloud(X, FX, keep), _as_cloud(Z, FZ, keep), keep


def cvo_evaluate(h, X, Z, T, FX=None, FZ=None) -> dict:
    cx, cz, keep = _clouds(X, Z, FX, FZ)
    Tm = _pose(T)
    e = Eval()
    _check(load_library().cvo_evaluate(h, ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data, ctypes.byref(e)))
    return dict(F=e.F, grad=np.array(e.grad[:]), hess=np.array(e.hess[:]).reshape(6, 6), i_theta=e.i_theta,
                pairs=int(e.pairs), candidates=int(e.candidates))


_GRAD_NAMES = ("dX", "dFX", "dZ", "dFZ")


def cvo_backward(h, X, Z, T, FX=None, FZ=None, dF=1.0, want=("dX", "dFX", "dZ", "dFZ", "dell")) -> dict:
    """Gradients of dF * F(T) with respect to the points, the features and the
    lengthscale (see cvo_backward in cvo.h).  Outputs are float32 torch CUDA
    tensors when X is a CUDA tensor, numpy arrays otherwise; names not in
    `want` are neither computed nor returned."""
    return _backward("cvo_backward", h, X, Z, T, FX, FZ, dF, want)


def cvo_metric_backward(h, X, Z, T, FX=None, FZ=None, di=1.0, want=("dX", "dFX", "dZ", "dFZ", "dell")) -> dict:
    """Gradients of di * i_theta (Eq. indicator_actual) with the outputs of
    cvo_backward (see cvo_metric_backward in cvo.h)."""
    return _backward("cvo_metric_backward", h, X, Z, T, FX, FZ, di, want)


def _backward(entry, h, X, Z, T, FX, FZ, dF, want) -> dict:
    cx, cz, keep = _clouds(X, Z, FX, FZ)
    Tm = _pose(T)
    D = 0
    for f in (FX, FZ):
        if f is not None and len(f.shape) == 2:
            D = int(f.shape[1])
    shapes = {"dX": (cx.n, 3), "dFX": (cx.n, D), "dZ": (cz.n, 3), "dFZ": (cz.n, D)}
    on_dev = bool(cx.on_device)
    out = {}
    ptrs = []
    for name in _GRAD_NAMES:
        if name not in want or (name in ("dFX", "dFZ") and D == 0):
            ptrs.append(None)
            continue
        if on_dev:
            torch = _torch()
            t = torch.empty(shapes[name], dtype=torch.float32, device=X.device)
            out[name] = t
            ptrs.append(t.data_ptr() if t.numel() else None)
        else:
            a = np.zeros(shapes[name], dtype=np.float32)
            out[name] = a
            ptrs.append(a.ctypes.data if a.size else None)
    dell = ctypes.c_double()
    _check(getattr(load_library(), entry)(h, ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data, float(dF), *ptrs,
                                          ctypes.byref(dell) if "dell" in want else None, int(on_dev)))
    if "dell" in want:
        out["dell"] = dell.value
    return out


def cvo_cosine(h, X, Z, T, FX=None, FZ=None, norms2=None):
    """Exact indicator of Eq. (indicator): returns (cos_theta, (|f_X|^2, |f_Z|^2)).
    Pass the returned norms back as norms2 to skip the two self sweeps."""
    cx, cz, keep = _clouds(X, Z, FX, FZ)
    Tm = _pose(T)
    nin = None if norms2 is None else np.ascontiguousarray(np.asarray(norms2, dtype=np.float64).reshape(2))
    nout = np.zeros(2)
    c = ctypes.c_double()
    _check(load_library().cvo_cosine(h, ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data,
                                     None if nin is None else nin.ctypes.data, ctypes.byref(c), nout.ctypes.data))
    return c.value, (float(nout[0]), float(nout[1]))


def cvo_cosine_dell(h, X, Z, T, FX=None, FZ=None):
    """The exact indicator of Eq. (indicator) and its derivative with respect
    to the lengthscale: returns (cos_theta, dcos/dl)."""
    cx, cz, keep = _clouds(X, Z, FX, FZ)
    Tm = _pose(T)
    c = ctypes.c_double()
    d = ctypes.c_double()
    _check(load_library().cvo_cosine_dell(h, ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data, ctypes.byref(c),
                                          ctypes.byref(d)))
    return c.value, d.value


def cvo_inner_product(h, X, Z, T, FX=None, FZ=None) -> float:
    cx, cz, keep = _clouds(X, Z, FX, FZ)
    Tm = _pose(T)
    out = ctypes.c_double()
    _check(load_library().cvo_inner_product(h, ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data, ctypes.byref(out)))
    return out.value


def cvo_gradient(h, X, Z, T, FX=None, FZ=None):
    cx, cz, keep = _clouds(X, Z, FX, FZ)
    Tm = _pose(T)
    g = np.zeros(6)
    F = ctypes.c_double()
    _check(load_library().cvo_gradient(h, ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data, g.ctypes.data,
                                       ctypes.byref(F)))
    return g, F.value


def cvo_metric(h, X, Z, T, FX=None, FZ=None) -> float:
    cx, cz, keep = _clouds(X, Z, FX, FZ)
    Tm = _pose(T)
    out = ctypes.c_double()
    _check(load_library().cvo_metric(h, ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data, ctypes.byref(out)))
    return out.value


def cvo_register_pair(h, X, Z, T_init, FX=None, FZ=None):
    cx, cz, keep = _clouds(X, Z, FX, FZ)
    T0 = _pose(T_init)
    Tout = np.zeros((4, 4))
    info = Info()
    rc = _check(load_library().cvo_register_pair(h, ctypes.byref(cx), ctypes.byref(cz), T0.ctypes.data,
                                                 Tout.ctypes.data, ctypes.byref(info)))
    d = info.as_dict()
    d["rc"] = rc
    return Tout, d


def _batch_clouds(pairs, keep):
    n = len(pairs)
    CX = (Cloud * max(n, 1))()
    CZ = (Cloud * max(n, 1))()
    T0 = np.zeros((max(n, 1), 4, 4))
    for k, (X, Z, T, FX, FZ) in enumerate(pairs):
        CX[k] = _as_cloud(X, FX, keep)
        CZ[k] = _as_cloud(Z, FZ, keep)
        T0[k] = _pose(T)
    return n, CX, CZ, T0


def cvo_register_batch(h, pairs):
    """pairs: sequence of (X, Z, T_init, FX, FZ)."""
    keep = []
    n, CX, CZ, T0 = _batch_clouds(pairs, keep)
    Tout = np.zeros_like(T0)
    infos = (Info * max(n, 1))()
    rc = _check(load_library().cvo_register_batch(h, n, CX, CZ, T0.ctypes.data, Tout.ctypes.data, infos))
    return Tout[:n], [infos[k].as_dict() for k in range(n)], rc


def cvo_register_sequence(h, frames, ell_first, T_first=None):
    """frames: sequence of (xyz, features) per frame.  Returns (T_rel
    (nframes-1, 4, 4), T_abs (nframes, 4, 4), infos, rc)."""
    keep = []
    n = len(frames)
    C = (Cloud * max(n, 1))()
    for k, (P, F) in enumerate(frames):
        C[k] = _as_cloud(P, F, keep)
    T_rel = np.zeros((max(n - 1, 1), 4, 4))
    T_abs = np.zeros((max(n, 1), 4, 4))
    infos = (Info * max(n - 1, 1))()
    T0 = None if T_first is None else _pose(T_first)
    rc = _check(load_library().cvo_register_sequence(h, n, C, float(ell_first), None if T0 is None else T0.ctypes.data,
                                                     T_rel.ctypes.data, T_abs.ctypes.data, infos))
    return T_rel[: max(n - 1, 0)], T_abs[:n], [infos[k].as_dict() for k in range(max(n - 1, 0))], rc


def cvo_shard_begin(h, X_rows, Z, n_total, T_init, FX_rows=None, FZ=None):
    """Starts an X-row shard of one registration (see cvo_shard_begin in cvo.h)."""
    cx, cz, keep = _clouds(X_rows, Z, FX_rows, FZ)
    T0 = _pose(T_init)
    return _check(load_library().cvo_shard_begin(h, ctypes.byref(cx), ctypes.byref(cz), int(n_total), T0.ctypes.data))


def cvo_shard_sweep(h, stats):
    """Queues the shard's sweep; stats: a float64 CUDA tensor of SHARD_STATS entries."""
    return _check(load_library().cvo_shard_sweep(h, ctypes.c_void_p(_stats_ptr(stats))))


def cvo_shard_step(h, stats, wait=False):
    """Queues the step from the summed statistics; with wait=True returns
    whether the registration has stopped (else None)."""
    done = ctypes.c_int(0)
    _check(load_library().cvo_shard_step(h, ctypes.c_void_p(_stats_ptr(stats)), ctypes.byref(done) if wait else None))
    return bool(done.value) if wait else None


def cvo_shard_end(h):
    Tout = np.zeros((4, 4))
    info = Info()
    rc = _check(load_library().cvo_shard_end(h, Tout.ctypes.data, ctypes.byref(info)))
    d = info.as_dict()
    d["rc"] = rc
    return Tout, d


def _stats_ptr(stats):
    torch = _torch()
    if torch is None or not isinstance(stats, torch.Tensor) or not stats.is_cuda:
        raise ValueError("stats must be a CUDA tensor")
    if stats.dtype != torch.float64 or stats.numel() != SHARD_STATS or not stats.is_contiguous():
        raise ValueError(f"stats must be a contiguous float64 tensor of {SHARD_STATS} entries")
    return stats.data_ptr()


def shard_rows(n, world, rank):
    """The rows [lo, hi) of an n-point cloud that shard `rank` of `world`
    holds: contiguous, disjoint, covering every row once, sizes differing by
    at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("need world >= 1, 0 <= rank < world and n >= 0")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def register_sharded(h, X_rows, Z, n_total, T_init, FX_rows=None, FZ=None, allreduce=None, *, max_iters,
                     check_every=8, stats=None):
    """Registers one pair whose X is split by rows over shards: this
    process holds the rows X_rows (of n_total) and all of Z.  Every
    iteration the shard's statistics go through allreduce (a callable that
    sums a float64 CUDA tensor over the shards in place, on the current
    stream, e.g. torch.distributed.all_reduce; None: this is the only
    shard), then the step, for at most max_iters iterations (the handle's
    params.max_iters).  Whether the registration has stopped is read every
    check_every iterations.  stats: the float64 CUDA tensor of SHARD_STATS
    entries to use (None: one is made).  Returns (T_out, info)."""
    torch = _torch()
    cvo_shard_begin(h, X_rows, Z, n_total, T_init, FX_rows, FZ)
    if stats is None:
        stats = torch.zeros(SHARD_STATS, dtype=torch.float64, device="cuda")
    for it in range(int(max_iters)):
        cvo_shard_sweep(h, stats)
        if allreduce is not None:
            allreduce(stats)
        wait = (it + 1) % check_every == 0
        if cvo_shard_step(h, stats, wait=wait):
            break
    return cvo_shard_end(h)


def cvo_get_trace(h, cap=100000) -> np.ndarray:
    out = np.zeros((max(cap, 1), TRACE_STRIDE))
    n = _check(load_library().cvo_get_trace(h, out.ctypes.data, cap))
    return out[: min(n, cap)].copy()


def cvo_set_timing(h, on=True):
    return _check(load_library().cvo_set_timing(h, int(bool(on))))


def cvo_set_tuning(h, cell_factor=0.5, super_delta=2):
    return _check(load_library().cvo_set_tuning(h, float(cell_factor), int(super_delta)))


def cvo_autotune(h, X, Z, T, FX=None, FZ=None) -> dict:
    """Times a registration of (X, Z) from pose T under a grid of tunings and
    keeps the fastest on the handle (see cvo_autotune in cvo.h)."""
    cx, cz, keep = _clouds(X, Z, FX, FZ)
    Tm = _pose(T)
    out = Tuning()
    _check(load_library().cvo_autotune(h, ctypes.byref(cx), ctypes.byref(cz), Tm.ctypes.data, ctypes.byref(out)))
    return out.as_dict()


def cvo_autotune_batch(h, pairs) -> dict:
    """Times a batched registration of pairs ((X, Z, T_init, FX, FZ) each)
    under a grid of tunings and keeps the fastest on the handle (see
    cvo_autotune_batch in cvo.h)."""
    keep = []
    n, CX, CZ, T0 = _batch_clouds(pairs, keep)
    out = Tuning()
    _check(load_library().cvo_autotune_batch(h, n, CX, CZ, T0.ctypes.data, ctypes.byref(out)))
    return out.as_dict()


LOOP_MODES = {"host": 0, "graph": 1, "persistent": 2}


def cvo_set_loop(h, mode):
    """Registration loop of a single pair: "graph" (default), "persistent" or "host"."""
    return _check(load_library().cvo_set_loop(h, LOOP_MODES[mode] if isinstance(mode, str) else int(mode)))


def cvo_inject_barrier_stall(h, barrier, poll_limit=4096):
    """Failure injection for the persistent loop's next registration (see
    cvo_inject_barrier_stall in cvo.h); barrier < 0 clears it."""
    return _check(load_library().cvo_inject_barrier_stall(h, int(barrier), int(poll_limit)))


def cvo_get_tuning(h) -> dict:
    out = Tuning()
    _check(load_library().cvo_get_tuning(h, ctypes.byref(out)))
    return out.as_dict()


def cvo_apply_tuning(h, cell_factor, super_delta, chunk_len, query_lanes=1):
    t = Tuning(float(cell_factor), int(super_delta), int(chunk_len), 0.0, int(query_lanes))
    return _check(load_library().cvo_apply_tuning(h, ctypes.byref(t)))


def cvo_sweep_time(h):
    ms = ctypes.c_double()
    n = ctypes.c_int()
    _check(load_library().cvo_sweep_time(h, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


class CVO:
    """A handle with fixed parameters (see make_params for the arguments)."""

    def __init__(self, stream=None, **kw):
        self.params = make_params(**kw)
        self.h = cvo_create(self.params, stream)

    def close(self):
        if self.h is not None:
            cvo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, **kw):
        self.params = make_params(**kw)
        cvo_set_params(self.h, self.params)

    def evaluate(self, X, Z, T, FX=None, FZ=None):
        return cvo_evaluate(self.h, X, Z, T, FX, FZ)

    def inner_product(self, X, Z, T, FX=None, FZ=None):
        return cvo_inner_product(self.h, X, Z, T, FX, FZ)

    def gradient(self, X, Z, T, FX=None, FZ=None):
        return cvo_gradient(self.h, X, Z, T, FX, FZ)

    def metric(self, X, Z, T, FX=None, FZ=None):
        return cvo_metric(self.h, X, Z, T, FX, FZ)

    def cosine(self, X, Z, T, FX=None, FZ=None, norms2=None):
        return cvo_cosine(self.h, X, Z, T, FX, FZ, norms2)

    def backward(self, X, Z, T, FX=None, FZ=None, dF=1.0, want=("dX", "dFX", "dZ", "dFZ", "dell")):
        return cvo_backward(self.h, X, Z, T, FX, FZ, dF, want)

    def register(self, X, Z, T_init=None, FX=None, FZ=None):
        return cvo_register_pair(self.h, X, Z, np.eye(4) if T_init is None else T_init, FX, FZ)

    def register_batch(self, pairs):
        return cvo_register_batch(self.h, pairs)

    def register_sequence(self, frames, ell_first, T_first=None):
        return cvo_register_sequence(self.h, frames, ell_first, T_first)

    def register_sharded(self, X_rows, Z, n_total, T_init=None, FX_rows=None, FZ=None, allreduce=None):
        return register_sharded(self.h, X_rows, Z, n_total, np.eye(4) if T_init is None else T_init, FX_rows, FZ,
                                allreduce, max_iters=self.params.max_iters)

    def trace(self):
        return cvo_get_trace(self.h)

    def autotune(self, X, Z, T=None, FX=None, FZ=None):
        return cvo_autotune(self.h, X, Z, np.eye(4) if T is None else T, FX, FZ)

    def autotune_batch(self, pairs):
        return cvo_autotune_batch(self.h, pairs)

    def tuning(self):
        return cvo_get_tuning(self.h)

    def set_loop(self, mode):
        return cvo_set_loop(self.h, mode)

    def apply_tuning(self, cell_factor, super_delta, chunk_len, query_lanes=1):
        return cvo_apply_tuning(self.h, cell_factor, super_delta, chunk_len, query_lanes)


# ---- differentiable form ---------------------------------------------------------

def _autograd_function(value_entry, grad_entry):
    """A torch.autograd.Function of a scalar of the double sum: value_entry
    computes it (cvo_inner_product or cvo_metric) and grad_entry its input
    gradients (cvo_backward or cvo_metric_backward), both in the library."""
    torch = _torch()
    if torch is None:  # pragma: no cover
        raise RuntimeError("the differentiable form needs PyTorch")

    class _Fn(torch.autograd.Function):
        """The scalar as a function of X, Z, their features and the
        lengthscale; the backward pass runs the library's gradient sweeps.
        T is a constant here: the pose gradient is cvo_gradient's se(3)
        vector."""

        @staticmethod
        def forward(ctx, X, Z, FX, FZ, ell, T, cvo):
            params = cvo.params
            ell_v = float(ell) if ell is not None else params.ell
            p = Params.from_buffer_copy(params)
            p.ell = ell_v
            cvo_set_params(cvo.h, p)
            try:
                v = value_entry(cvo.h, X, Z, T, FX, FZ)
            finally:
                cvo_set_params(cvo.h, params)
            ctx.cvo = cvo
            ctx.T = np.array(_pose(T))
            ctx.ell = ell_v
            ctx.save_for_backward(X, Z, FX, FZ)
            ctx.ell_meta = (ell.dtype, ell.device) if isinstance(ell, torch.Tensor) else None
            dev = X.device if isinstance(X, torch.Tensor) else "cpu"
            return torch.tensor(v, dtype=torch.float64, device=dev)

        @staticmethod
        def backward(ctx, gF):
            X, Z, FX, FZ = ctx.saved_tensors
            need = ctx.needs_input_grad
            want = [n for n, k in (("dX", 0), ("dZ", 1), ("dFX", 2), ("dFZ", 3)) if need[k]]
            if need[4]:
                want.append("dell")
            if not want:
                return (None,) * 7
            cvo = ctx.cvo
            params = cvo.params
            p = Params.from_buffer_copy(params)
            p.ell = ctx.ell
            cvo_set_params(cvo.h, p)
            try:
                out = grad_entry(cvo.h, X, Z, ctx.T, FX, FZ, float(gF), tuple(want))
            finally:
                cvo_set_params(cvo.h, params)

            def as_grad(name, like):
                if name not in out:
                    return None
                g = out[name]
                if not isinstance(g, torch.Tensor):
                    g = torch.from_numpy(g)
                return g.to(dtype=like.dtype, device=like.device)

            dell = None
            if "dell" in out and ctx.ell_meta is not None:
                dell = torch.tensor(out["dell"], dtype=ctx.ell_meta[0], device=ctx.ell_meta[1])
            return (as_grad("dX", X), as_grad("dZ", Z), as_grad("dFX", FX) if FX is not None else None,
                    as_grad("dFZ", FZ) if FZ is not None else None, dell, None, None)

    return _Fn


_fn_cache = {}


def CVOInnerProduct():
    """The torch.autograd.Function class of the differentiable F (built on
    first use so that importing this package does not need PyTorch)."""
    if "F" not in _fn_cache:
        _fn_cache["F"] = _autograd_function(cvo_inner_product, cvo_backward)
    return _fn_cache["F"]


def CVOMetric():
    """The torch.autograd.Function class of the differentiable indicator of
    Eq. (indicator_actual) (value from cvo_metric, gradients from
    cvo_metric_backward)."""
    if "metric" not in _fn_cache:
        _fn_cache["metric"] = _autograd_function(cvo_metric, cvo_metric_backward)
    return _fn_cache["metric"]


def inner_product_fn(cvo: "CVO", X, Z, T, FX=None, FZ=None, ell=None):
    """Differentiable F(T) (a float64 scalar tensor) of torch tensors X (N, 3),
    Z (M, 3), features FX, FZ and an optional lengthscale tensor ell (else the
    handle's params.ell); gradients flow to every input that requires them."""
    return CVOInnerProduct().apply(X, Z, FX, FZ, ell, T, cvo)


def metric_fn(cvo: "CVO", X, Z, T, FX=None, FZ=None, ell=None):
    """Differentiable indicator i_theta of Eq. (indicator_actual), with the
    arguments of inner_product_fn."""
    return CVOMetric().apply(X, Z, FX, FZ, ell, T, cvo)


def _cosine_function():
    torch = _torch()
    if torch is None:  # pragma: no cover
        raise RuntimeError("the differentiable form needs PyTorch")

    class _Cos(torch.autograd.Function):
        """The exact indicator of Eq. (indicator) as a function of the
        lengthscale (the clouds, features and pose are constants here); the
        value and dcos/dl come from cvo_cosine_dell."""

        @staticmethod
        def forward(ctx, ell, X, Z, FX, FZ, T, cvo):
            p = Params.from_buffer_copy(cvo.params)
            p.ell = float(ell)
            cvo_set_params(cvo.h, p)
            try:
                c, d = cvo_cosine_dell(cvo.h, X, Z, T, FX, FZ)
            finally:
                cvo_set_params(cvo.h, cvo.params)
            ctx.d = d
            return torch.tensor(c, dtype=ell.dtype, device=ell.device)

        @staticmethod
        def backward(ctx, g):
            return g * ctx.d, None, None, None, None, None, None

    return _Cos


def cosine_fn(cvo: "CVO", X, Z, T, FX=None, FZ=None, ell=None):
    """Differentiable exact indicator cos_theta(l) of Eq. (indicator): ell is
    a scalar tensor (requires_grad for dcos/dl); the clouds, features and
    pose are held constant."""
    if "cos" not in _fn_cache:
        _fn_cache["cos"] = _cosine_function()
    torch = _torch()
    if ell is None:
        ell = torch.tensor(cvo.params.ell, dtype=torch.float64)
    return _fn_cache["cos"].apply(ell, X, Z, FX, FZ, T, cvo)
