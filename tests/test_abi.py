"""The C ABI library builds for sm_103a, loads, and exports every entry
point that include/vcm.h declares (no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "vcm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vcm_[a-z_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_1310_7297_gb300 import build as B
    from paper_1310_7297_gb300 import vcm

    path = B.build()
    names = declared()
    assert len(names) >= 15
    # the product library and the checked build (VCM_CHECKED) alike
    for p in (path, B.LIB_CHECKED):
        L = ctypes.CDLL(p)
        for n in names:
            assert hasattr(L, n), (p, n)
    assert sorted(vcm.EXPORTS) == names


def test_struct_layouts_match_header(tmp_path):
    """ctypes layouts equal what a C compiler makes of include/vcm.h."""
    import subprocess

    from paper_1310_7297_gb300 import vcm

    structs = {"vcm_request": vcm.vcm_request, "vcm_stats": vcm.vcm_stats, "vcm_result": vcm.vcm_result,
               "vcm_tune": vcm.vcm_tune, "vcm_memory": vcm.vcm_memory}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vcm.h"', "int main(void){"]
    for name, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines.append("return 0;}")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)])
    got = dict(l.split() for l in subprocess.check_output([str(exe)]).decode().splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (name, f)]) == getattr(cls, f).offset, (name, f)


def test_create_without_gpu_fails_cleanly():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1310_7297_gb300 import VcmError, Context

    with pytest.raises(VcmError) as e:
        Context(0)
    assert e.value.status == -4   # VCM_E_CUDA


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    from paper_1310_7297_gb300 import vcm

    monkeypatch.setattr(vcm, "_lib", None)
    monkeypatch.setattr(vcm, "LIB_PATH", str(tmp_path / "nope.so"))
    with pytest.raises(RuntimeError):
        vcm.lib()
