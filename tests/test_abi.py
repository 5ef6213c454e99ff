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


def _table(gj, n, ncols, key_type=0, col_type=0, fake=0x1000):
    t = gj.Table()
    t.key_type, t.ncols, t.n = key_type, ncols, n
    t.key = fake if n else None
    for c in range(ncols):
        t.col_type[c] = col_type
        t.cols[c] = fake + 64 * (c + 1) if n else None
    return t


def test_argument_checks_run_before_any_device_work(lib):
    """Invalid arguments are rejected on the host (GJ_ERR_INVALID_ARG = 1,
    GJ_ERR_UNSUPPORTED = 2) before any CUDA call, so these run without a GPU.
    The pointers are never dereferenced."""
    from paper_2312_00720_gb300 import gj
    R, S = _table(gj, 10, 1), _table(gj, 20, 1)
    T = _table(gj, 20, 2)
    cnt = ctypes.c_void_p(0x2000)
    o = gj.Options()
    lib.gj_options_default(ctypes.byref(o))
    join = lambda R, S, o, T, cap: lib.gj_join(ctypes.byref(R), ctypes.byref(S), ctypes.byref(o), ctypes.byref(T),
                                                ctypes.c_int64(cap), cnt, None)
    o.join_variant = 8  # past GJ_JOIN_PHJ_MN
    assert join(R, S, o, T, 20) == 1
    lib.gj_options_default(ctypes.byref(o))
    o.radix_bits = 17
    assert join(R, S, o, T, 20) == 1
    lib.gj_options_default(ctypes.byref(o))
    assert join(R, _table(gj, 20, 1, key_type=1), o, T, 20) == 1  # key types differ
    assert join(R, S, o, _table(gj, 20, 3), 20) == 1  # T has the wrong column count
    T9 = _table(gj, 20, 8)
    T9.ncols = 9  # R.ncols + S.ncols = 9: more columns than a gj_table holds
    assert join(_table(gj, 10, 5), _table(gj, 20, 4), o, T9, 20) == 1
    assert join(R, S, o, T, -1) == 1
    assert join(_table(gj, 1 << 31, 1), S, o, T, 20) == 2  # more rows than supported

    ops = (ctypes.c_int32 * 2)(0, 1)
    cols = (ctypes.c_int32 * 2)(0, 0)
    outs = (ctypes.c_void_p * 2)(0x3000, 0x4000)
    gb = lambda t, nagg, ops, o: lib.gj_groupby(ctypes.byref(t), nagg, ops, cols, ctypes.byref(o),
                                                 ctypes.c_void_p(0x5000), outs, ctypes.c_int64(8), cnt, None)
    o.groupby_variant = 7  # past GJ_GB_SGB_DE
    assert gb(R, 2, ops, o) == 1
    lib.gj_options_default(ctypes.byref(o))
    assert gb(R, 0, ops, o) == 1
    assert gb(R, 2, (ctypes.c_int32 * 2)(0, 9), o) == 1  # unknown aggregate
    assert lib.gj_groupby(ctypes.byref(R), 2, (ctypes.c_int32 * 2)(0, 0), (ctypes.c_int32 * 2)(0, 3),
                          ctypes.byref(o), ctypes.c_void_p(0x5000), outs, ctypes.c_int64(8), cnt, None) == 1

    # the allocation-free partition: more than 8 bits in its one pass is unsupported
    out = _table(gj, 10, 1)
    assert lib.gj_radix_partition_noalloc(ctypes.byref(R), 0, 9, 0, ctypes.byref(out), None, 0, None) == 2
    assert lib.gj_radix_partition_noalloc(ctypes.byref(R), 4, 4, 0, ctypes.byref(out), None, 0, None) == 1


def test_binding_variant_codes_match_the_header():
    """The Python names of the join / group-by variants carry the enum values
    include/gj.h declares."""
    from paper_2312_00720_gb300 import gj
    text = open(os.path.join(ROOT, "include", "gj.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    enum = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(GJ_(?:JOIN|GB)_\w+)\s*=\s*(\d+)", text)}
    for name, code in gj.JOIN.items():
        assert enum["GJ_JOIN_" + name.upper()] == code, name
    for name, code in gj.GROUPBY.items():
        assert enum["GJ_GB_" + name.upper()] == code, name
    assert len([k for k in enum if k.startswith("GJ_JOIN_")]) == len(gj.JOIN)
    assert len([k for k in enum if k.startswith("GJ_GB_")]) == len(gj.GROUPBY)


def test_heuristic_choice_matches_the_oracle_rules(lib):
    """The library's rule-based variant choice (gj_heuristic_choose, host code)
    agrees with the oracle's statement of the paper's join rule and group-by
    decision tree over a grid of hints. The library sizes HGB's shared memory
    as 8 bytes per aggregate under a 200 KB budget when the device does not
    report a smaller one."""
    import itertools
    from oracle import heuristics as hz
    from paper_2312_00720_gb300 import gj
    jcode = {hz.JOIN_PHJ_TR: gj.JOIN["phj_tr"], hz.JOIN_PHJ_UR: gj.JOIN["phj_ur"]}
    gcode = {hz.GB_HGB: gj.GROUPBY["hgb"], hz.GB_SGB: gj.GROUPBY["sgb"], hz.GB_PGB: gj.GROUPBY["pgb"]}
    for mr, z, kb, groups, nagg in itertools.product((0.1, 0.24, 0.25, 1.0), (0.0, 0.49, 0.5, 1.0, 1.25), (4, 8),
                                                     (4, 2560, 2561, 1 << 20), (1, 10)):
        jv, gv = gj.heuristic_choose(1 << 20, 1 << 22, kb, 2, 2, nagg, z, mr, groups)
        assert jv == jcode[hz.choose_join(mr, z, kb)], (mr, z, kb)
        assert gv == gcode[hz.choose_groupby(groups, 8 * nagg, 200 * 1024, z, kb)], (groups, nagg, z)


def test_query_features_follow_the_header(lib):
    """gj_query_features (host code) writes the 12 raw features include/gj.h lists."""
    import math
    from paper_2312_00720_gb300 import gj
    for nr, ns, kb, cr, cs, nagg, z, mr, g in [(1 << 20, 1 << 22, 4, 2, 3, 4, 0.5, 0.25, 1 << 12),
                                               (1000, 10, 8, 1, 8, 10, 0.0, 1.0, 7), (0, 5, 4, 1, 1, 1, 1.25, 0.1, 1)]:
        f = gj.query_features(nr, ns, kb, cr, cs, nagg, z, mr, g)
        want = [math.log2(nr + 1), math.log2(ns + 1), kb, cr, cs, z, mr, math.log2(g + 1), nagg,
                math.log2((nr + 1) / (ns + 1)), 4 * cs, math.log2(g + 1) / math.log2(ns + 2)]
        assert f.tolist() == pytest.approx(want, rel=1e-6, abs=1e-6)


def test_binding_refuses_host_tensors(lib):
    """The binding has no CPU path: host tensors are refused before any library call."""
    import torch
    from paper_2312_00720_gb300 import gj
    k = torch.arange(16, dtype=torch.int32)
    v = [torch.zeros(16, dtype=torch.int32)]
    with pytest.raises(ValueError, match="CUDA"):
        gj.join(k, v, k, v, variant="phj_tr")
    with pytest.raises(ValueError, match="CUDA"):
        gj.groupby(k, v, ["count"], [0], variant="sgb")
    with pytest.raises(ValueError, match="CUDA"):
        gj.join_groupby(k, v, k, v, (0, 0, 4), ["count"], [(1, 0, 0)])
    with pytest.raises(ValueError, match="CUDA"):
        gj.radix_partition(k, v, 0, 4)


def test_selector_set_validates_on_the_host(lib):
    """gj_selector_set copies host arrays; a missing normaliser or a non-positive
    standard deviation is an argument error, NULL theta removes the network."""
    import numpy as np
    theta = np.zeros(5707, dtype=np.float32)
    mean = np.zeros(12, dtype=np.float32)
    std = np.ones(12, dtype=np.float32)
    f = lib.gj_selector_set
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    assert f(theta.ctypes.data, None, std.ctypes.data) == 1
    bad = std.copy()
    bad[7] = 0.0
    assert f(theta.ctypes.data, mean.ctypes.data, bad.ctypes.data) == 1
    bad[7] = np.nan
    assert f(theta.ctypes.data, mean.ctypes.data, bad.ctypes.data) == 1
    assert f(theta.ctypes.data, mean.ctypes.data, std.ctypes.data) == 0
    assert f(None, None, None) == 0
