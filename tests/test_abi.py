"""The C-ABI library loads without a GPU and exports every entry point that
include/amrvac_gb300.h declares; the Python binding names the same calls."""
import ctypes
import os
import re

import pytest

from paper_2004_03275_gb300 import amrvac, build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "amrvac_gb300.h")


def declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ("amr_create", "amr_set_state", "amr_step", "amr_regrid", "amr_read_state", "mg_create",
                 "mg_solve", "rd_step"):
        assert must in names


def test_library_exports_every_declared_symbol():
    if not os.path.exists(build.LIB):
        build.build()
    lib = ctypes.CDLL(build.LIB)
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    assert set(declared()) <= set(amrvac.exported_symbols())


def test_load_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(amrvac, "_lib", None)
    with pytest.raises(RuntimeError):
        amrvac.load()


def test_build_flags_keep_parity_and_target_sm103a():
    """Every unit compiles for sm_103a only; the float64 units (compared with the oracle to
    1e-12) are compiled without multiply-add contraction, the float32 stage units with fast math."""
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    srcs = build.sources()
    assert srcs and all(s.endswith(".cu") for s in srcs)
    for s in srcs:
        flags = build.unit_flags(s)
        if s.startswith(("euler_f64", "mg_f64")):
            assert flags == ["--fmad=false"], s
        elif s.startswith("euler_f32"):
            assert flags == ["--use_fast_math"], s
        else:
            assert "--use_fast_math" not in flags, s
    assert {"euler_f64_1d.cu", "euler_f64_2d.cu", "euler_f64_3d.cu", "mg_f64_tree.cu"} <= set(srcs)
