"""The C-ABI library loads and exports every entry point the header declares (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hicu.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hicu_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2004_08962_gb300 import build, hicu
    build.build()
    return hicu.lib()


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("hicu_gram", "hicu_nullspace", "hicu_conv_null", "hicu_conv_null_adjoint",
              "hicu_gd_step", "hicu_reconstruct"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2004_08962_gb300 import hicu
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", hicu.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (hicu_\w+)", out))
    assert set(declared_functions()) <= exported
    assert set(hicu.EXPORTED) == set(declared_functions())


def test_build_targets_sm103a_only():
    from paper_2004_08962_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_host_only_queries(lib):
    from paper_2004_08962_gb300 import hicu
    g = hicu.make_geom((64, 48, 1), 4, (5, 5, 1))
    assert hicu.hicu_filter_length(g) == 100
    assert hicu.hicu_num_outputs(g, hicu.make_region((0, 0, 0), (64, 48, 1))) == 60 * 44
    assert hicu.hicu_num_outputs(g, hicu.make_region((4, 4, 0), (16, 16, 1))) == 12 * 12
    # region larger than the array, or smaller than the kernel -> -1
    assert hicu.hicu_num_outputs(g, hicu.make_region((10, 0, 0), (64, 48, 1))) == -1
    assert hicu.hicu_num_outputs(g, hicu.make_region((0, 0, 0), (4, 48, 1))) == -1
    gc = hicu.make_geom((8, 6, 5), 2, (3, 3, 3), circular=(0, 0, 1))
    assert hicu.hicu_num_outputs(gc, hicu.make_region((0, 0, 0), (8, 6, 5))) == 6 * 4 * 5
    bad = hicu.make_geom((8, 6, 5), 0, (3, 3, 3))
    assert hicu.hicu_filter_length(bad) == -1
    assert lib.hicu_status_string(6) == b"HICU_ERR_TIMEOUT"
