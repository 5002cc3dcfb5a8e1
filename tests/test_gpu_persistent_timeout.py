"""The persistent registration loop's bounded grid barriers, made to run
out on purpose without a fault: cvo_inject_barrier_stall makes one block of
the next persistent registration leave the kernel at a chosen grid barrier
instead of arriving, with a short poll limit.  Every other block gives up
waiting, the kernel returns, and the call reports CVO_ERR_TIMEOUT; nothing
hangs, and the handle registers correctly afterwards (the same result as a
fresh handle, bitwise)."""
import numpy as np
import pytest

import scenes

torch = pytest.importorskip("torch")
import paper_2012_03683_gb300 as cvo  # noqa: E402

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda")


@pytest.fixture(scope="module")
def pair():
    p = scenes.street_pair()
    sel = np.random.Generator(np.random.PCG64(23)).permutation(p.n)[:5000]
    args = (dev(p.X[sel]), dev(p.Z[sel]), np.eye(4), dev(p.FX[sel]), dev(p.FZ[sel]))
    kw = dict(blocks=p.blocks, ell=0.3, ell_min=0.05, cutoff_mult=3.0, max_iters=30, anneal=True)
    return args, kw


@pytest.mark.parametrize("barrier", [0, 1, 5])
def test_a_stalled_barrier_gives_up_and_the_handle_recovers(pair, barrier):
    args, kw = pair
    with cvo.CVO(**kw) as fresh:
        fresh.set_loop("persistent")
        T_ref, info_ref = fresh.register(*args)
    with cvo.CVO(**kw) as h:
        h.set_loop("persistent")
        cvo.cvo_inject_barrier_stall(h.h, barrier, 4096)
        with pytest.raises(cvo.CvoError) as e:
            h.register(*args)
        assert e.value.status == cvo.Status.ERR_TIMEOUT
        assert "barrier" in str(e.value)
        # the injection holds for one registration: the next one completes
        T, info = h.register(*args)
        assert np.array_equal(T, T_ref) and info["iters"] == info_ref["iters"]
        # and the other loop modes are unaffected by a pending injection
        cvo.cvo_inject_barrier_stall(h.h, barrier, 4096)
        h.set_loop("graph")
        Tg, _ = h.register(*args)
        cvo.cvo_inject_barrier_stall(h.h, -1, 0)
    with cvo.CVO(**kw) as g:
        Tg_ref, _ = g.register(*args)
    assert np.array_equal(Tg, Tg_ref)
