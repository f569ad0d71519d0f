"""The C-ABI library builds for sm_103a, loads, and exports every symbol include/stdg.h declares.

CPU-only: no call here launches GPU work (argument validation happens before
any CUDA call, and context creation without a GPU returns STDG_ERR_CUDA)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stdg.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2201_05800_gb300 import build, stdg
    build.build()
    return stdg.load()


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stdg_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "stdg_create" in names and "stdg_advance_slab" in names
    for n in names:
        assert hasattr(lib, n), n


def test_struct_layout_matches_header(lib):
    """stdg_config_default fills the ctypes mirror with the documented defaults (the layout itself
    is compared with the C header by test_struct_offsets_match_the_c_header)."""
    from paper_2201_05800_gb300 import stdg
    d = stdg.config_default()
    assert d.dim == 1 and d.N == 3 and d.s == 3 and d.gmres_m == 30
    assert abs(d.newton_rtol - 1e-10) < 1e-25 and abs(d.gamma - 1.4) < 1e-15
    # natural alignment of the C struct: 4 ints, 6 doubles, 3 ints, 3 doubles ... ends in a size_t
    assert ctypes.sizeof(stdg.stdg_config_desc) % 8 == 0


def test_invalid_configs_rejected_without_gpu(lib):
    from paper_2201_05800_gb300 import stdg
    bad = [dict(dim=4), dict(N=0), dict(N=8), dict(s=1), dict(s=6), dict(dt=-1.0), dict(gmres_m=0),
           dict(gmres_m=64), dict(equation=7), dict(equation=2, dim=3), dict(cells=[0, 1, 1]),
           dict(predictor=2), dict(predictor=-1), dict(precond=3), dict(viscosity=-1.0)]
    for kw in bad:
        d = stdg.make_config(**kw)
        h = ctypes.c_void_p()
        st = lib.stdg_create(ctypes.byref(d), None, ctypes.byref(h))
        assert st == 1, kw
        assert not h.value


def test_make_config_rejects_unknown_fields(lib):
    from paper_2201_05800_gb300 import stdg
    with pytest.raises(KeyError):
        stdg.make_config(predicter=1)


def test_status_strings(lib):
    from paper_2201_05800_gb300 import stdg
    for k in range(10):
        assert stdg.status_string(k)
    assert stdg.version().startswith("stdg-gb300")


def test_create_without_gpu_reports_cuda_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2201_05800_gb300 import stdg
    with pytest.raises(stdg.StdgError) as e:
        stdg.Context(stdg.make_config())
    assert e.value.status == 3


def test_null_arguments(lib):
    assert lib.stdg_create(None, None, None) == 1
    assert lib.stdg_destroy(None) == 1
    assert lib.stdg_state_len(None) == 0


def test_batch_validation_without_gpu(lib):
    from paper_2201_05800_gb300 import stdg
    h = ctypes.c_void_p()
    assert lib.stdg_batch_create(None, None, ctypes.byref(h)) == 1
    for bad in [stdg.stdg_batch_desc(3, stdg.EULER, 4, 1 << 20), stdg.stdg_batch_desc(2, stdg.EULER, 0, 1 << 20),
                stdg.stdg_batch_desc(2, stdg.EULER, 4, 0), stdg.stdg_batch_desc(1, stdg.BURGERS, 4, 1 << 20)]:
        assert lib.stdg_batch_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
        assert not h.value
    assert lib.stdg_batch_destroy(None) == 1
    assert lib.stdg_batch_free_bytes(None) == 0


def test_server_without_gpu(lib):
    """Server creation validates its arguments first, then reports the missing device as a
    status (no worker thread is left behind)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2201_05800_gb300 import stdg
    h = ctypes.c_void_p()
    bad = stdg.stdg_batch_desc(2, stdg.EULER, 0, 1 << 20)
    assert lib.stdg_server_create(ctypes.byref(bad), 4, ctypes.byref(h)) == 1
    ok = stdg.stdg_batch_desc(2, stdg.EULER, 4, 1 << 20)
    assert lib.stdg_server_create(ctypes.byref(ok), 0, ctypes.byref(h)) == 1
    assert lib.stdg_server_create(ctypes.byref(ok), 4, ctypes.byref(h)) == 3
    assert not h.value
    assert lib.stdg_server_destroy(None) == 1


def test_struct_offsets_match_the_c_header(tmp_path):
    """Size and every field offset of the ctypes mirrors equal those of the C structs, from a C
    probe compiled against include/stdg.h (catches a field added on one side only)."""
    import shutil
    import subprocess
    from paper_2201_05800_gb300 import stdg
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    mirrors = {"stdg_config_desc": stdg.stdg_config_desc, "stdg_slab_stats": stdg.stdg_slab_stats,
               "stdg_profile": stdg.stdg_profile, "stdg_batch_desc": stdg.stdg_batch_desc}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "stdg.h"', "int main(void) {"]
    for name, cls in mirrors.items():
        lines.append('  printf("%s size %%zu\\n", sizeof(%s));' % (name, name))
        for f, _ in cls._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));' % (name, f, name, f))
    lines += ["  return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "probe"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for name, cls in mirrors.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert got[(name, f)] == getattr(cls, f).offset, (name, f)
