"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/mkgb.h declares; the ctypes structs have the header's layout.  No GPU needed
(no compute call is made)."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2312_11728_gb300 import build as B
from paper_2312_11728_gb300 import mkgb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mkgb.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mkgb.load_library()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mkgb_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_entry_point_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    assert set(names) == set(mkgb.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (mkgb_\w+)", out))
    for n in names:
        assert n in exported, n
        assert hasattr(lib, n)


def test_every_entry_point_has_its_argument_types(lib):
    """The binding declares each entry point's parameters, as many as the header gives it: an
    undeclared pointer parameter would go through ctypes as a 32-bit int and lose the high bits of
    any host address above 2 GB."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for n in mkgb.EXPORTS:
        m = re.search(r"\b" + n + r"\s*\(([^)]*)\)", text)
        assert m, n
        params = m.group(1).strip()
        count = 0 if params in ("", "void") else params.count(",") + 1
        assert getattr(lib, n).argtypes is not None, n
        assert len(getattr(lib, n).argtypes) == count, (n, count)


def test_library_is_built_for_sm_103a_only(lib):
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert B.up_to_date()


def test_version_and_null_context(lib):
    assert b"sm_103a" in lib.mkgb_version()
    assert lib.mkgb_last_error(None) == b"null context"
    assert lib.mkgb_build(None, None, 0) == -1


def test_struct_layouts_match_the_header(tmp_path):
    probe = tmp_path / "probe.c"
    probe.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mkgb.h"\n'
                     'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(mkgb_layer), sizeof(mkgb_params),'
                     ' sizeof(mkgb_tracks), offsetof(mkgb_layer, n_eta_bins), offsetof(mkgb_tracks, max_plan));'
                     'return 0;}\n')
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(probe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    assert got == [C.sizeof(mkgb.Layer), C.sizeof(mkgb.Params), C.sizeof(mkgb.Tracks),
                   mkgb.Layer.n_eta_bins.offset, mkgb.Tracks.max_plan.offset]


def test_binding_refuses_mixed_host_and_device_arrays():
    import numpy as np
    with pytest.raises(mkgb.MkgbError):
        mkgb._same(True, False)
    with pytest.raises(mkgb.MkgbError):
        mkgb._ptr(np.zeros(3, np.float64), np.float32, out=True)
