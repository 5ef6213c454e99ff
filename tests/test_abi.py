"""The C-ABI library loads on a machine without a GPU and exports every entry
point declared in include/*.h (no compute calls here)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(gj_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2312_00720_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_operators():
    names = declared_functions()
    for f in ("gj_join", "gj_groupby", "gj_join_groupby", "gj_radix_partition", "gj_status_string",
              "gj_get_device_status", "gj_set_allocator", "gj_options_default"):
        assert f in names


def test_every_declared_symbol_is_exported(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_host_only_helpers(lib):
    lib.gj_status_string.restype = ctypes.c_char_p
    assert lib.gj_status_string(5) == b"GJ_ERR_DUPLICATE_KEY"
    assert lib.gj_status_string(99) == b"GJ_UNKNOWN_STATUS"
    from paper_2312_00720_gb300 import gj
    o = gj.Options()
    lib.gj_options_default(ctypes.byref(o))
    assert o.join_variant == 0 and o.sync == 0 and o.zipf_hint < 0


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_2312_00720_gb300 import gj
    monkeypatch.setattr(gj, "_lib", None)
    monkeypatch.setattr(gj, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError):
        gj.load()
