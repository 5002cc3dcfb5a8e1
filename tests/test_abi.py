"""The C ABI library builds, loads and exports every entry point that
include/cvo.h declares, and the binding's ctypes structures have the header's
layout.  No compute call is made: these tests run without a GPU."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2012_03683_gb300 as cvo
from paper_2012_03683_gb300 import build as cvo_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cvo.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cvo_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("cvo_create", "cvo_destroy", "cvo_register_pair", "cvo_register_batch", "cvo_inner_product",
                     "cvo_gradient", "cvo_metric", "cvo_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(cvo_build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_and_reports_version():
    cvo.load_library()
    assert "sm_103a" in cvo.cvo_version()
    assert cvo.cvo_last_error() == ""


def test_invalid_params_rejected_without_gpu_work():
    p = cvo.make_params(ell=-1.0)
    with pytest.raises(cvo.CvoError) as e:
        cvo.cvo_create(p, stream=0)
    assert e.value.status == cvo.Status.ERR_INVALID_ARG
    assert "ell" in cvo.cvo_last_error()
    p = cvo.make_params(blocks=[("se", 3, 0.0, 1.0)])
    with pytest.raises(cvo.CvoError):
        cvo.cvo_create(p, stream=0)
    p = cvo.make_params(anneal=True, ell=0.1, ell_min=0.2)
    with pytest.raises(cvo.CvoError):
        cvo.cvo_create(p, stream=0)


def test_struct_layout_matches_header(tmp_path):
    """Compile a host-only C probe of the header and compare sizes/offsets."""
    src = tmp_path / "probe.c"
    src.write_text(r'''
#include <stddef.h>
#include <stdio.h>
#include "cvo.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(cvo_feat_block), sizeof(cvo_cloud), sizeof(cvo_params),
         sizeof(cvo_info), sizeof(cvo_eval));
  printf("%zu %zu %zu %zu %zu\n", offsetof(cvo_params, blocks), offsetof(cvo_params, max_iters),
         offsetof(cvo_params, max_step_trans), offsetof(cvo_params, feat_cutoff_mult), offsetof(cvo_info, pairs));
  printf("%zu %zu\n", offsetof(cvo_cloud, feat_dtype), offsetof(cvo_eval, candidates));
  printf("%zu %zu %zu\n", sizeof(cvo_tuning), offsetof(cvo_tuning, chunk_len), offsetof(cvo_tuning, measured_ms));
  return 0;
}
''')
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in out]
    got = [ctypes.sizeof(cvo.FeatBlock), ctypes.sizeof(cvo.Cloud), ctypes.sizeof(cvo.Params),
           ctypes.sizeof(cvo.Info), ctypes.sizeof(cvo.Eval),
           cvo.Params.blocks.offset, cvo.Params.max_iters.offset, cvo.Params.max_step_trans.offset,
           cvo.Params.feat_cutoff_mult.offset, cvo.Info.pairs.offset, cvo.Cloud.feat_dtype.offset, cvo.Eval.candidates.offset,
           ctypes.sizeof(cvo.Tuning), cvo.Tuning.chunk_len.offset, cvo.Tuning.measured_ms.offset]
    assert vals == got


def test_every_field_offset_matches_header(tmp_path):
    """Every field of every structure the binding mirrors sits at the
    header's offset (a C probe prints offsetof for each ctypes field name)."""
    structs = {"cvo_feat_block": cvo.FeatBlock, "cvo_cloud": cvo.Cloud, "cvo_params": cvo.Params,
               "cvo_info": cvo.Info, "cvo_tuning": cvo.Tuning, "cvo_eval": cvo.Eval}
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "cvo.h"', 'int main(void) {']
    expected = []
    for cname, ct in structs.items():
        lines.append(f'  printf("%zu\\n", sizeof({cname}));')
        expected.append(ctypes.sizeof(ct))
        for fname, _ in ct._fields_:
            lines.append(f'  printf("%zu\\n", offsetof({cname}, {fname}));')
            expected.append(getattr(ct, fname).offset)
    lines += ['  return 0;', '}']
    src = tmp_path / "fields.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "fields"
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expected
