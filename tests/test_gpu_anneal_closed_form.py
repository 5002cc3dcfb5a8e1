"""The library's annealing trigger and stopping test on the closed-form
registration problems of tests/anneal_closed_form.py (one axial pair,
translated; two point-symmetric pairs, rotated), through cvo_register_pair.

The GPU must take every decision the closed form takes -- the iterations at
which the lengthscale decays (Sec. IV) and the iteration at which the run
stops -- and agree with the FP64 oracle on the same float32 inputs: each
iteration's lengthscale (both update it in FP64), the indicator
(Eq. indicator_actual, relative 1e-5) and the final pose (1e-4 rad / m,
here far tighter).  Every decision of these cases is at least 2 % of the
tolerance away from its threshold, so the FP32 sums cannot flip one.
"""
import math

import numpy as np
import pytest

import anneal_closed_form as acf
import oracle

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu

C_ELL, C_ITH, C_DEC = 0, 2, 8


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


@pytest.mark.parametrize("loop", ["graph", "persistent"])
@pytest.mark.parametrize("case", sorted(acf.CASES))
def test_gpu_annealing_and_stop_match_the_closed_form(case, loop):
    X, Z, kw = acf.points(case)
    X, Z = _f32(X), _f32(Z)          # the library takes float32 coordinates
    ref = acf.trajectory(**acf.CASES[case])
    n_ref, decays_ref = acf.summary(ref)

    h = cvo.CVO(**kw)
    h.set_loop(loop)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Zd = torch.tensor(Z, dtype=torch.float32, device="cuda")
    T, info = h.register(Xd, Zd, np.eye(4))
    tr = h.trace()
    h.close()

    assert info["status"] == 0 and info["iters"] == n_ref == tr.shape[0]
    assert list(np.nonzero(tr[:, C_DEC])[0]) == decays_ref

    To, io, tro = oracle.register(X, Z, np.eye(4), **kw)
    assert io["iters"] == n_ref and list(np.nonzero(tro[:, 8])[0]) == decays_ref
    assert np.array_equal(tr[:, C_ELL], tro[:, C_ELL])
    assert np.allclose(tr[:, C_ITH], tro[:, C_ITH], rtol=1e-5, atol=0.0)
    assert info["ell_final"] == io["ell_final"]
    D = np.linalg.inv(T) @ To
    rot = math.acos(max(-1.0, min(1.0, (np.trace(D[:3, :3]) - 1.0) / 2.0)))
    assert rot < 1e-6 and np.linalg.norm(D[:3, 3]) < 1e-6
