"""Host logic of the Python binding that needs no GPU: how point clouds,
feature rows, poses and parameters are marshalled into the C structures
(pointer, count, device flag, feature dtype), which inputs it refuses, and
that the buffers it passes stay alive and hold the caller's values."""
import ctypes

import numpy as np
import pytest

import paper_2012_03683_gb300 as cvo
from paper_2012_03683_gb300 import _as_cloud, _pose

torch = pytest.importorskip("torch")


def read_floats(ptr, count):
    return np.ctypeslib.as_array((ctypes.c_float * count).from_address(ptr)).copy()


def read_u16(ptr, count):
    return np.ctypeslib.as_array((ctypes.c_uint16 * count).from_address(ptr)).copy()


def test_numpy_points_become_contiguous_float32():
    X = np.arange(12, dtype=np.float64).reshape(4, 3) * 0.5
    keep = []
    c = _as_cloud(X, None, keep)
    assert c.n == 4 and c.on_device == 0 and not c.feat
    assert np.array_equal(read_floats(c.xyz, 12), X.astype(np.float32).ravel())
    # a flat array of 3N values is read as N rows; a strided view is copied
    flat = _as_cloud(X.ravel(), None, keep)
    assert flat.n == 4
    Xt = np.asfortranarray(X)
    ct = _as_cloud(Xt, None, keep)
    assert np.array_equal(read_floats(ct.xyz, 12), X.astype(np.float32).ravel())


def test_numpy_features_float32_or_bfloat16_bits():
    X = np.zeros((3, 3), np.float32)
    F = np.array([[0.25, 0.5], [1.0, 2.0], [3.0, -1.0]])
    keep = []
    c = _as_cloud(X, F, keep)
    assert c.feat_dtype == 0 and np.array_equal(read_floats(c.feat, 6), F.astype(np.float32).ravel())
    bits = np.array([[0x3F80, 0x4000], [0x4040, 0x4080], [0xBF80, 0x0000]], dtype=np.uint16)
    cb = _as_cloud(X, bits, keep)
    assert cb.feat_dtype == 1 and np.array_equal(read_u16(cb.feat, 6), bits.ravel())


def test_empty_cloud_passes_null_pointers():
    keep = []
    c = _as_cloud(np.zeros((0, 3), np.float32), np.zeros((0, 4), np.float32), keep)
    assert c.n == 0 and not c.xyz and not c.feat


def test_torch_cpu_tensors():
    X = torch.arange(9, dtype=torch.float32).reshape(3, 3)
    F = torch.tensor([[1.0, 2.0], [3.0, 4.0], [5.0, 6.0]], dtype=torch.bfloat16)
    keep = []
    c = _as_cloud(X, F, keep)
    assert c.n == 3 and c.on_device == 0 and c.feat_dtype == 1
    assert np.array_equal(read_floats(c.xyz, 9), X.numpy().ravel())
    assert np.array_equal(read_u16(c.feat, 6), F.view(torch.int16).numpy().astype(np.uint16).ravel())
    # a transposed (non-contiguous) view is made contiguous and kept alive
    Xt = torch.arange(9, dtype=torch.float32).reshape(3, 3).t()
    ct = _as_cloud(Xt, None, keep)
    assert np.array_equal(read_floats(ct.xyz, 9), Xt.contiguous().numpy().ravel())
    assert any(k.data_ptr() == ct.xyz for k in keep if isinstance(k, torch.Tensor))


def test_torch_inputs_refused():
    keep = []
    with pytest.raises(ValueError):
        _as_cloud(torch.zeros(4, 3, dtype=torch.float64), None, keep)
    with pytest.raises(ValueError):
        _as_cloud(torch.zeros(4, 2), None, keep)
    with pytest.raises(ValueError):
        _as_cloud(torch.zeros(4, 3), torch.zeros(4, 2, dtype=torch.float16), keep)


def test_pose_and_params():
    T = np.eye(4, dtype=np.float32)
    T[0, 3] = 0.5
    P = _pose(T)
    assert P.dtype == np.float64 and P.flags.c_contiguous and P[0, 3] == 0.5
    with pytest.raises(ValueError):
        _pose(np.eye(3))
    p = cvo.make_params(blocks=[("se", 3, 0.2, 1.5), ("dot", 19, 1.0, 1.0)], ell=0.3, ell_min=0.05,
                        cutoff_mult=2.5, anneal=True, feat_cutoff_mult=1.6)
    assert p.n_blocks == 2 and p.blocks[0].kind == 0 and p.blocks[1].kind == 1 and p.blocks[1].dim == 19
    assert p.blocks[0].scale == pytest.approx(0.2) and p.blocks[0].sigma == pytest.approx(1.5)
    assert (p.ell, p.ell_min, p.cutoff_mult, p.anneal, p.feat_cutoff_mult) == (0.3, 0.05, 2.5, 1, 1.6)
    assert cvo.make_params(ell=0.2).ell_min == 0.2          # no floor given: the floor is ell
    with pytest.raises(ValueError):
        cvo.make_params(blocks=[("se", 1, 0.2, 1.0)] * 5)
    with pytest.raises(KeyError):
        cvo.make_params(blocks=[("cosine", 3, 0.2, 1.0)])


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library, and with no way to build it, every call
    raises: there is no fallback."""
    import paper_2012_03683_gb300 as pkg

    def no_build():
        raise RuntimeError("nvcc failed (stand-in)")

    monkeypatch.setattr(pkg, "_lib", None)
    monkeypatch.setattr(pkg._build, "LIB", str(tmp_path / "libcvo.so"))
    monkeypatch.setattr(pkg._build, "build", no_build)
    with pytest.raises(RuntimeError, match="not built"):
        pkg.load_library(build_if_missing=False)
    with pytest.raises(RuntimeError, match="stand-in"):
        pkg.CVO(ell=0.1)
    with pytest.raises(RuntimeError, match="stand-in"):
        pkg.cvo_version()
