"""The C ABI library builds, loads and exports every declared entry point, and
the Python binding's structs have the C layout.  No GPU is needed."""
import ctypes
import os
import subprocess

import pytest

import paper_2405_10565_gb300 as hr
from paper_2405_10565_gb300 import _lib
from paper_2405_10565_gb300.build import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _lib.header_functions()
    assert len(names) >= 20
    raw = ctypes.CDLL(_lib.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing
    # and the binding covers every declared function
    assert set(names) <= set(_lib._SIGS)


def test_struct_layout_matches_c(tmp_path, lib):
    src = tmp_path / "sz.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "hairrt.h"\n'
        "int main(void){printf(\"%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n\","
        "sizeof(hr_camera), sizeof(hr_light), sizeof(hr_render_desc), sizeof(hr_stats),"
        "sizeof(hr_hair_desc), sizeof(hr_request), sizeof(hr_result),"
        "offsetof(hr_render_desc, seed), offsetof(hr_render_desc, precision),"
        "offsetof(hr_request, rgb_out), sizeof(hr_tile_record),"
        "offsetof(hr_stats, refined_entries), offsetof(hr_stats, heavy_tiles));return 0;}\n")
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = [int(v) for v in subprocess.check_output([str(exe)]).split()]
    want = [ctypes.sizeof(_lib.hr_camera), ctypes.sizeof(_lib.hr_light),
            ctypes.sizeof(_lib.hr_render_desc), ctypes.sizeof(_lib.hr_stats),
            ctypes.sizeof(_lib.hr_hair_desc), ctypes.sizeof(_lib.hr_request),
            ctypes.sizeof(_lib.hr_result), _lib.hr_render_desc.seed.offset,
            _lib.hr_render_desc.precision.offset, _lib.hr_request.rgb_out.offset,
            ctypes.sizeof(_lib.hr_tile_record), _lib.hr_stats.refined_entries.offset,
            _lib.hr_stats.heavy_tiles.offset]
    assert got == want


def test_no_device_reports_cuda_error(lib):
    # on a host without a GPU the library must refuse, not fall back
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hr.HairRTError) as ei:
        hr.hr_create(0)
    assert ei.value.status == hr.HR_ECUDA


def test_missing_library_fails_loudly(tmp_path):
    with pytest.raises(RuntimeError):
        _lib._lib = None
        try:
            _lib.load(str(tmp_path / "nope.so"))
        finally:
            _lib._lib = None


def test_header_constants_match_the_binding():
    """Every #define HR_* value and hr_status code of hairrt.h equals the
    binding's constant of the same name (a flag added on one side only would
    otherwise pass unseen)."""
    import re
    text = open(os.path.join(ROOT, "include", "hairrt.h")).read()
    defines = dict(re.findall(r"^#define (HR_[A-Z0-9_]+) (\d+)u?\b", text, re.M))
    assert len(defines) >= 15
    for name, value in defines.items():
        assert hasattr(_lib, name), name
        assert getattr(_lib, name) == int(value), name
    codes = dict(re.findall(r"^\s+(HR_E?[A-Z]+) = (\d+),?", text, re.M))
    assert codes.get("HR_OK") == "0" and len(codes) >= 8, codes
    for name, value in codes.items():
        assert getattr(_lib, name) == int(value), name
