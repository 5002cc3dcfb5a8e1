"""BF16 feature storage: the error of each result against the FP64 oracle,
split into arithmetic error (oracle fed the same BF16-rounded features) and
storage error (oracle fed the FP32 features).

Bounds: the arithmetic error obeys the FP32 parity tolerances (F relative
1e-5, gradient 1e-4 of |g| plus the FP32 rounding floor); the storage error
is set by the BF16 rounding of the features (relative 2^-9 per entry): the
colour exponent (u - v)^2 / (2 l_c^2) moves by about 2^-8 (u - v)^2 / l_c^2
and each label inner product by at most 2^-8 of itself, so F and g move by
well under 1 %.  The test prints every measured error."""
import numpy as np
import pytest

import oracle
import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(a)).to("cuda")
    return t.to(dtype) if dtype is not None else t


def workloads():
    s = scenes.street_pair()
    r = scenes.room_pair()
    b = scenes.batch_pairs(n_pairs=2)[1]
    return [("street-20k", s, 0.3, 3.0), ("room-19k", r, 0.1, 3.0), ("batch-pair", b, 0.1, 3.0)]


@pytest.mark.parametrize("idx", [0, 1, 2])
def test_bf16_error_per_result(idx):
    name, p, ell, cm = workloads()[idx]
    FX32 = np.asarray(p.FX, np.float32)
    FZ32 = np.asarray(p.FZ, np.float32)
    kw = dict(blocks=p.blocks, ell=ell, cutoff_mult=cm)
    h = cvo.CVO(**kw)
    T = p.T_true
    X, Z = dev(p.X), dev(p.Z)
    ref32 = oracle.evaluate(p.X, p.Z, T, FX=FX32, FZ=FZ32, **kw)
    ref16 = oracle.evaluate(p.X, p.Z, T, FX=scenes.bf16_round(FX32), FZ=scenes.bf16_round(FZ32), **kw)
    g32 = h.evaluate(X, Z, T, dev(FX32), dev(FZ32))
    g16 = h.evaluate(X, Z, T, dev(FX32, torch.bfloat16), dev(FZ32, torch.bfloat16))

    def errs(got, ref):
        gn = np.linalg.norm(ref["g"])
        return abs(got["F"] - ref["F"]) / abs(ref["F"]), np.abs(got["grad"] - ref["g"]).max() / gn

    f32_f, f32_g = errs(g32, ref32)
    ar_f, ar_g = errs(g16, ref16)
    st_f, st_g = errs(g16, ref32)
    print(f"\n[{name}] f32 features: F rel {f32_f:.2e}, grad {f32_g:.2e} of |g|; "
          f"bf16 features: arithmetic F rel {ar_f:.2e}, grad {ar_g:.2e}; "
          f"vs f32 oracle F rel {st_f:.2e}, grad {st_g:.2e}")
    floor16 = 1e-7 * ref16["gscale"] / np.linalg.norm(ref16["g"])
    floor32 = 1e-7 * ref32["gscale"] / np.linalg.norm(ref32["g"])
    assert f32_f <= 1e-5 and f32_g <= 1e-4 + floor32
    assert ar_f <= 1e-5 and ar_g <= 1e-4 + floor16
    assert st_f <= 1e-2 and st_g <= 5e-2
