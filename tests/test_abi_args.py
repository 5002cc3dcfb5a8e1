"""Host-side argument checks of the C ABI: every entry point given a NULL
handle or a NULL output returns CVO_ERR_INVALID_ARG with a message (and
cvo_destroy accepts NULL, as the header states); creating a handle where no
GPU is present fails with CVO_ERR_CUDA and a message instead of crashing;
the allocation-free entry point rejects what it cannot evaluate before it
touches the device.  No kernel is launched: these run without a GPU."""
import ctypes

import pytest

import paper_2012_03683_gb300 as cvo

INVALID = cvo.Status.ERR_INVALID_ARG


@pytest.fixture(scope="module")
def lib():
    return cvo.load_library()


def last_error():
    return cvo.cvo_last_error()


def expect_invalid(rc, fragment):
    assert rc == INVALID, (rc, last_error())
    assert fragment in last_error(), last_error()


def test_null_handle_rejected_by_every_entry_point(lib):
    d = ctypes.c_double(0.0)
    i = ctypes.c_int(0)
    grad = (ctypes.c_double * 6)()
    T = (ctypes.c_double * 16)()
    params = cvo.make_params()
    tun = cvo.Tuning(0.5, 2, 64, 0.0)
    ev = cvo.Eval()
    info = cvo.Info()
    ref = ctypes.byref
    calls = {
        "cvo_set_params": lambda: lib.cvo_set_params(None, ref(params)),
        "cvo_evaluate": lambda: lib.cvo_evaluate(None, None, None, T, ref(ev)),
        "cvo_inner_product": lambda: lib.cvo_inner_product(None, None, None, T, ref(d)),
        "cvo_metric": lambda: lib.cvo_metric(None, None, None, T, ref(d)),
        "cvo_gradient": lambda: lib.cvo_gradient(None, None, None, T, grad, None),
        "cvo_backward": lambda: lib.cvo_backward(None, None, None, T, 1.0, None, None, None, None, ref(d), 0),
        "cvo_metric_backward": lambda: lib.cvo_metric_backward(None, None, None, T, 1.0, None, None, None, None,
                                                               ref(d), 0),
        "cvo_cosine": lambda: lib.cvo_cosine(None, None, None, T, None, ref(d), None),
        "cvo_cosine_dell": lambda: lib.cvo_cosine_dell(None, None, None, T, ref(d), ref(d)),
        "cvo_register_pair": lambda: lib.cvo_register_pair(None, None, None, T, T, ref(info)),
        "cvo_register_batch": lambda: lib.cvo_register_batch(None, 1, None, None, T, T, None),
        "cvo_register_sequence": lambda: lib.cvo_register_sequence(None, 2, None, 0.3, None, None, None, None),
        "cvo_get_trace": lambda: lib.cvo_get_trace(None, None, 0),
        "cvo_set_tuning": lambda: lib.cvo_set_tuning(None, 0.5, 2),
        "cvo_autotune": lambda: lib.cvo_autotune(None, None, None, T, ref(tun)),
        "cvo_autotune_batch": lambda: lib.cvo_autotune_batch(None, 1, None, None, T, ref(tun)),
        "cvo_get_tuning": lambda: lib.cvo_get_tuning(None, ref(tun)),
        "cvo_apply_tuning": lambda: lib.cvo_apply_tuning(None, ref(tun)),
        "cvo_set_loop": lambda: lib.cvo_set_loop(None, 1),
        "cvo_inject_barrier_stall": lambda: lib.cvo_inject_barrier_stall(None, 1, 100),
        "cvo_set_timing": lambda: lib.cvo_set_timing(None, 1),
        "cvo_sweep_time": lambda: lib.cvo_sweep_time(None, ref(d), ref(i)),
    }
    for name, call in calls.items():
        rc = call()
        assert rc == INVALID, (name, rc)
        assert "NULL" in last_error(), (name, last_error())
    assert lib.cvo_destroy(None) == cvo.Status.OK


def test_null_outputs_rejected_before_the_handle_is_used(lib):
    """The output pointer is checked before anything else: with both the
    handle and the output NULL, the message names the output."""
    T = (ctypes.c_double * 16)()
    expect_invalid(lib.cvo_inner_product(None, None, None, T, None), "F is NULL")
    expect_invalid(lib.cvo_metric(None, None, None, T, None), "i_theta is NULL")
    expect_invalid(lib.cvo_gradient(None, None, None, T, None, None), "grad is NULL")


def test_create_rejects_a_null_output(lib):
    p = cvo.make_params()
    expect_invalid(lib.cvo_create(ctypes.byref(p), None, None), "out is NULL")


def test_create_without_a_device_fails_cleanly(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: creation succeeds there")
    p = cvo.make_params()
    h = ctypes.c_void_p(12345)
    rc = lib.cvo_create(ctypes.byref(p), None, ctypes.byref(h))
    assert rc == cvo.Status.ERR_CUDA, (rc, last_error())
    assert "cudaGetDevice" in last_error()
    assert h.value is None        # the output handle is cleared on failure
    with pytest.raises(cvo.CvoError) as e:
        cvo.CVO(ell=0.1)
    assert e.value.status == cvo.Status.ERR_CUDA


def test_noalloc_rejects_before_device_work(lib):
    fn = lib.cvo_evaluate_dense_noalloc
    fn.restype = ctypes.c_int
    T = (ctypes.c_double * 16)(*[1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1])
    X = cvo.Cloud()
    out = ctypes.c_void_p(16)     # never dereferenced: every call below fails its checks first
    ref = ctypes.byref

    def call(p):
        return fn(ref(p) if p is not None else None, None, ref(X), ref(X), T, out)

    expect_invalid(call(None), "NULL argument")
    expect_invalid(call(cvo.make_params(cutoff_mult=3.0)), "dense sum only")
    expect_invalid(call(cvo.make_params(cutoff_mult=0.0, ell=0.0)), "ell and sigma")
    expect_invalid(call(cvo.make_params(cutoff_mult=0.0, sigma=-1.0)), "ell and sigma")
    wide = [("dot", 19, 1.0, 1.0), ("se", 3, 0.2, 1.0), ("dot", 5, 1.0, 1.0)]   # 27 entries > 24
    expect_invalid(call(cvo.make_params(cutoff_mult=0.0, blocks=wide)), "24 feature entries")
    bad = cvo.make_params(cutoff_mult=0.0, blocks=[("se", 3, 0.2, 1.0)])
    bad.blocks[0].scale = 0.0
    expect_invalid(call(bad), "invalid feature block")
    # the same checks as cvo_create: a finite scale and a finite sigma
    bad.blocks[0].scale = float("inf")
    expect_invalid(call(bad), "invalid feature block")
    bad.blocks[0].scale = 0.2
    bad.blocks[0].sigma = float("nan")
    expect_invalid(call(bad), "invalid feature block")
    with pytest.raises(cvo.CvoError) as e:
        cvo.cvo_create(bad, stream=0)
    assert e.value.status == INVALID


C_CLIENT = r'''
#include <stdio.h>
#include "cvo.h"

int main(void)
{
    cvo_params p = {0};
    p.ell = 0.3; p.ell_min = 0.3; p.sigma = 1.0; p.cutoff_mult = 3.0; p.max_iters = 20;
    p.decay = 0.98; p.indicator_tol = 1e-3; p.step_tol_rot = 1e-5; p.step_tol_trans = 1e-5;
    p.max_step_rot = 0.1;
    cvo_handle h;
    cvo_status s = cvo_create(&p, NULL, &h);
    if (s != CVO_OK) {
        printf("create failed: %d: %s\n", (int)s, cvo_last_error());
        return 3;
    }
    const float X[6] = {0.f, 0.f, 0.f, 0.5f, 0.f, 0.f}, Z[6] = {0.02f, 0.f, 0.f, 0.52f, 0.f, 0.f};
    cvo_cloud cx = {X, 2, NULL, CVO_F32, 0}, cz = {Z, 2, NULL, CVO_F32, 0};
    const double I[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
    double T[16];
    cvo_info info;
    s = cvo_register_pair(h, &cx, &cz, I, T, &info);
    cvo_destroy(h);
    printf("register: %d, %d iterations, t_x = %.6f\n", (int)s, info.iters, T[3]);
    return s < 0 ? 4 : 0;
}
'''


def test_c_client_builds_and_runs(lib, tmp_path):
    """A plain C program includes the header, links the library with gcc and
    runs: without a GPU it gets CVO_ERR_CUDA and a message from cvo_create;
    with one, the two-point registration moves Z onto X (t_x = -0.02)."""
    import os
    import subprocess
    from paper_2012_03683_gb300 import build as cvo_build
    so = cvo_build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    src = tmp_path / "client.c"
    src.write_text(C_CLIENT)
    exe = tmp_path / "client"
    libdir = os.path.dirname(so)
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(root, "include"), str(src),
                    "-L", libdir, "-lcvo", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        assert r.returncode == 0, r.stdout + r.stderr
        t_x = float(r.stdout.strip().rsplit("=", 1)[1])
        assert t_x == pytest.approx(-0.02, abs=1e-4)
    else:
        assert r.returncode == 3, r.stdout + r.stderr
        assert "create failed: -2" in r.stdout and "cudaGetDevice" in r.stdout
