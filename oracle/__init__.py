"""CPU oracle for the join / group-by path -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. The product path (the CUDA library and its Python
binding) never calls it and shares no code with it.

Contents
  * ``oracle.cpp`` (loaded here through ctypes): single-threaded join, two
    independent group-bys (hash map / sort), join -> group-by, and the stable
    radix-partition permutation -- Sec. 2.2, 2.3 and Algorithm 1 of the paper.
  * ``cost_models``: the paper's cost models M2 (Sec. 4.1.3), M3 (Sec. 4.1.4)
    and M4 (Sec. 4.4), pinned to the printed "Estimated" series.
  * ``heuristics``: the join rule of Sec. 5.1.10 (join summary) / Sec. 7 and the group-by
    decision tree (Fig. groupby-dt).
  * ``mlp``: float64 forward/backward of the variant-selector network and its
    SGD and Adam updates.

Parity status: every function here is pinned by tests under ``tests/`` (brute
force, invariants, closed forms, the paper's printed numbers; the MLP by central
finite differences, an affine special case, and Adam's closed forms: the first
step from zero moments and every step of a constant gradient move each parameter
by lr * g / (|g| + eps)); none is unpinned.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")

AGG_SUM, AGG_COUNT, AGG_MIN, AGG_MAX = 0, 1, 2, 3
_AGG_NAMES = {"sum": AGG_SUM, "count": AGG_COUNT, "min": AGG_MIN, "max": AGG_MAX}


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so next to it (plain g++, -O2, no threads)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, i32, p = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        lib.oracle_join.restype = i64
        lib.oracle_join.argtypes = [p, p, i64, i32, p, p, i64, i32, p, i64]
        for fn in (lib.oracle_groupby_hash, lib.oracle_groupby_sort):
            fn.restype = i64
            fn.argtypes = [p, p, i64, i32, p, p, p, i64]
        lib.oracle_join_groupby.restype = i64
        lib.oracle_join_groupby.argtypes = [p, p, i64, i32, p, p, i64, i32, i32, i32, i64, i32, p, p, p, p, i64]
        lib.oracle_radix_partition.restype = None
        lib.oracle_radix_partition.argtypes = [p, i64, i32, i32, i32, i32, p, p]
        _lib = lib
    return _lib


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a).astype(np.int64, copy=False))


def _ptrs(cols):
    arrs = [_i64(c) for c in cols]
    tab = (ctypes.c_void_p * max(1, len(arrs)))(*[a.ctypes.data for a in arrs])
    return arrs, tab


def _ops(aggs):
    ops = np.array([_AGG_NAMES[a] if isinstance(a, str) else int(a) for a in aggs], dtype=np.int32)
    return ops


def join(rkey, rcols, skey, scols) -> np.ndarray:
    """T(key, r.., s..) as an int64 matrix, one row per match (S order, then R order)."""
    lib = _load()
    rk, sk = _i64(rkey), _i64(skey)
    ra, rt = _ptrs(rcols)
    sa, st = _ptrs(scols)
    w = 1 + len(ra) + len(sa)
    m = lib.oracle_join(rk.ctypes.data, rt, len(rk), len(ra), sk.ctypes.data, st, len(sk), len(sa), None, 0)
    out = np.empty((m, w), dtype=np.int64)
    lib.oracle_join(rk.ctypes.data, rt, len(rk), len(ra), sk.ctypes.data, st, len(sk), len(sa),
                    out.ctypes.data, m)
    return out


def _groupby(fn, key, cols, aggs, agg_cols):
    lib = _load()
    k = _i64(key)
    ca, ct = _ptrs(cols)
    ops = _ops(aggs)
    oc = np.asarray(agg_cols, dtype=np.int32)
    out = np.empty((max(1, len(k)), 1 + len(ops)), dtype=np.int64)
    g = getattr(lib, fn)(k.ctypes.data, ct, len(k), len(ops), ops.ctypes.data, oc.ctypes.data,
                         out.ctypes.data, len(out))
    return out[:g].copy()


def groupby_hash(key, cols, aggs, agg_cols) -> np.ndarray:
    """A(k, a1..) via a hash map, groups in first-occurrence order."""
    return _groupby("oracle_groupby_hash", key, cols, aggs, agg_cols)


def groupby_sort(key, cols, aggs, agg_cols) -> np.ndarray:
    """A(k, a1..) via std::stable_sort and a scan of equal-key runs, ascending keys."""
    return _groupby("oracle_groupby_sort", key, cols, aggs, agg_cols)


def join_groupby(rkey, rcols, skey, scols, *, g_side: int, g_col: int, g_mod: int, aggs, agg_side, agg_col):
    """GROUP BY (side.col % g_mod) over R join S; aggregate j over column agg_col[j] of agg_side[j]."""
    lib = _load()
    rk, sk = _i64(rkey), _i64(skey)
    ra, rt = _ptrs(rcols)
    sa, st = _ptrs(scols)
    ops = _ops(aggs)
    asd = np.asarray(agg_side, dtype=np.int32)
    acl = np.asarray(agg_col, dtype=np.int32)
    # the number of groups never exceeds the number of join rows; size from the join count
    m = lib.oracle_join(rk.ctypes.data, rt, len(rk), len(ra), sk.ctypes.data, st, len(sk), len(sa), None, 0)
    out = np.empty((max(1, m), 1 + len(ops)), dtype=np.int64)
    g = lib.oracle_join_groupby(rk.ctypes.data, rt, len(rk), len(ra), sk.ctypes.data, st, len(sk), len(sa),
                                g_side, g_col, g_mod, len(ops), ops.ctypes.data, asd.ctypes.data,
                                acl.ctypes.data, out.ctypes.data, len(out))
    return out[:g].copy()


def radix_partition(key, key_bytes: int, lo: int, hi: int, transform: int = 0):
    """Stable radix-partition permutation and partition offsets on bits [lo, hi) (offsets: None above 24 bits)."""
    lib = _load()
    k = _i64(key)
    perm = np.empty(len(k), dtype=np.int64)
    offs = np.empty((1 << (hi - lo)) + 1, dtype=np.int64) if hi - lo <= 24 else None
    lib.oracle_radix_partition(k.ctypes.data, len(k), key_bytes, lo, hi, transform, perm.ctypes.data,
                               None if offs is None else offs.ctypes.data)
    return perm, offs


def gather(src, index) -> np.ndarray:
    """The gather primitive (Sec. 2.3): out[i] = src[index[i]]."""
    src = np.asarray(src)
    return np.array([src[int(j)] for j in np.asarray(index)], dtype=src.dtype)


def canonical(rows: np.ndarray) -> np.ndarray:
    """Rows sorted lexicographically by all columns (signed int64): the comparison form."""
    rows = np.asarray(rows, dtype=np.int64)
    if rows.ndim != 2 or rows.shape[0] == 0:
        return rows.reshape(-1, rows.shape[-1] if rows.ndim == 2 else 0)
    order = np.lexsort(rows.T[::-1])
    return rows[order]
