"""Python binding of libgj (include/gj.h): argument marshalling only.

Every entry point takes torch CUDA tensors, fills the C descriptors with their
device pointers and calls the library on torch's current stream. Outputs are
allocated with torch.empty on the same device. There is no fallback: if
libgj.so is missing or fails to load, ``load()`` raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libgj.so")

MAX_COLS = 8
MAX_AGGS = 32
I32, I64 = 0, 1
AGG = {"sum": 0, "count": 1, "min": 2, "max": 3}
JOIN = {"auto": 0, "phj_tr": 1, "phj_ur": 2, "nphj": 3, "nphj_mn": 4, "smj_tr": 5, "smj_ur": 6, "phj_mn": 7}
GROUPBY = {"auto": 0, "hgb": 1, "sgb": 2, "pgb": 3, "sgb_ur": 4, "pgb_ur": 5, "sgb_de": 6}
STATUS = {0: "GJ_OK", 1: "GJ_ERR_INVALID_ARG", 2: "GJ_ERR_UNSUPPORTED", 3: "GJ_ERR_OOM", 4: "GJ_ERR_CAPACITY",
          5: "GJ_ERR_DUPLICATE_KEY", 6: "GJ_ERR_TIMEOUT", 7: "GJ_ERR_CUDA"}


class GjError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}")


class Table(ctypes.Structure):
    _fields_ = [("key_type", ctypes.c_int32), ("ncols", ctypes.c_int32), ("n", ctypes.c_int64),
                ("key", ctypes.c_void_p), ("col_type", ctypes.c_int32 * MAX_COLS),
                ("cols", ctypes.c_void_p * MAX_COLS)]


class Options(ctypes.Structure):
    _fields_ = [("join_variant", ctypes.c_int32), ("groupby_variant", ctypes.c_int32),
                ("selector", ctypes.c_int32), ("radix_bits", ctypes.c_int32), ("bits_per_pass", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("sync", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("zipf_hint", ctypes.c_float), ("match_ratio_hint", ctypes.c_float),
                ("groups_hint", ctypes.c_int64)]


SELECT = {"heuristic": 0, "mlp": 1, "cost": 2}


class CostParams(ctypes.Structure):
    _fields_ = [("bg_over_br", ctypes.c_double), ("bg_over_bl2", ctypes.c_double), ("l2_bytes", ctypes.c_double),
                ("smem_bytes", ctypes.c_double), ("launch_bytes", ctypes.c_double), ("sync_bytes", ctypes.c_double),
                ("hot_row_bytes", ctypes.c_double), ("num_sms", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ColRef(ctypes.Structure):
    _fields_ = [("side", ctypes.c_int32), ("col", ctypes.c_int32), ("modulus", ctypes.c_int64)]


_lib = None


def load():
    """Load libgj.so (built by paper_2312_00720_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
    lib = ctypes.CDLL(LIB_PATH)
    p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    P = ctypes.POINTER
    lib.gj_options_default.argtypes = [P(Options)]
    lib.gj_options_default.restype = None
    lib.gj_status_string.argtypes = [i32]
    lib.gj_status_string.restype = ctypes.c_char_p
    lib.gj_get_device_status.argtypes = [p]
    lib.gj_get_device_status.restype = i32
    lib.gj_set_allocator.argtypes = [p, p, p]
    lib.gj_set_allocator.restype = i32
    lib.gj_radix_partition.argtypes = [P(Table), i32, i32, i32, P(Table), p, P(Options), p]
    lib.gj_radix_partition.restype = i32
    lib.gj_join.argtypes = [P(Table), P(Table), P(Options), P(Table), i64, p, p]
    lib.gj_join.restype = i32
    lib.gj_groupby.argtypes = [P(Table), i32, p, p, P(Options), p, p, i64, p, p]
    lib.gj_groupby.restype = i32
    lib.gj_join_groupby.argtypes = [P(Table), P(Table), ColRef, i32, p, p, P(Options), p, p, i64, p, p]
    lib.gj_join_groupby.restype = i32
    lib.gj_profile_enable.argtypes = [i32]
    lib.gj_profile_enable.restype = None
    lib.gj_profile_read.argtypes = [p, p, i32]
    lib.gj_profile_read.restype = i32
    lib.gj_kernel_name.argtypes = [i32]
    lib.gj_kernel_name.restype = ctypes.c_char_p
    lib.gj_kernel_launches.argtypes = []
    lib.gj_kernel_launches.restype = i64
    lib.gj_gather.argtypes = [p, i64, i32, p, i64, p, P(Options), p]
    lib.gj_gather.restype = i32
    lib.gj_set_wait_limit.argtypes = [ctypes.c_uint64]
    lib.gj_set_wait_limit.restype = i32
    lib.gj_check_bounded_wait.argtypes = [i32, p]
    lib.gj_check_bounded_wait.restype = i32
    _lib = lib
    return lib


# C types of the scratch allocator hooks (gj_set_allocator)
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_hooks = None  # keeps the installed ctypes callbacks alive


def set_allocator(alloc=None, free=None):
    """Installs Python scratch-allocator hooks (gj_set_allocator): alloc(bytes,
    stream) returns a device address or 0 (the call then fails with GJ_ERR_OOM),
    free(ptr, stream) releases one. No arguments restores the library's own
    stream-ordered allocations."""
    global _hooks
    lib = load()
    if alloc is None:
        _raise(lib.gj_set_allocator(None, None, None), "gj_set_allocator")
        _hooks = None
        return
    a = ALLOC_FN(lambda nbytes, stream, ctx: alloc(int(nbytes), stream) or None)
    f = FREE_FN(lambda ptr, stream, ctx: free(int(ptr), stream))
    _raise(lib.gj_set_allocator(ctypes.cast(a, ctypes.c_void_p), ctypes.cast(f, ctypes.c_void_p), None),
           "gj_set_allocator")
    _hooks = (a, f)


def gather(src: torch.Tensor, index: torch.Tensor, *, sync: bool = True, out=None) -> torch.Tensor:
    """gj_gather: out[i] = src[index[i]] (int32 or int64 src, int32 index)."""
    if src.dtype not in (torch.int32, torch.int64) or index.dtype != torch.int32:
        raise TypeError("src int32/int64, index int32")
    _check_dev(src, src.numel())
    _check_dev(index, index.numel())
    if out is None:
        out = torch.empty(index.numel(), dtype=src.dtype, device=src.device)
    o = options(sync=sync)
    _raise(load().gj_gather(src.data_ptr(), src.numel(), src.element_size(), index.data_ptr(), index.numel(),
                            out.data_ptr(), ctypes.byref(o), _stream()), "gj_gather")
    return out


def set_wait_limit(ns: int):
    """Wait limit of the library's bounded device-side waits on the current
    device, in nanoseconds (0 = the default of 2 s)."""
    _raise(load().gj_set_wait_limit(int(ns)), "gj_set_wait_limit")


def check_bounded_wait(kind: int) -> int:
    """Runs bounded wait `kind` (0 look-back, 1 mbarrier, 2 task counter) on a flag
    nothing sets; returns the status the kernel recorded (6 = GJ_ERR_TIMEOUT)."""
    return int(load().gj_check_bounded_wait(kind, _stream()))


BATCH_MAX_AGGS = 8


class Query(ctypes.Structure):
    _fields_ = [("R", Table), ("S", Table), ("group_key", ColRef), ("nagg", ctypes.c_int32),
                ("ops", ctypes.c_int32 * BATCH_MAX_AGGS), ("agg_cols", ColRef * BATCH_MAX_AGGS),
                ("out_keys", ctypes.c_void_p), ("out_aggs", ctypes.c_void_p * BATCH_MAX_AGGS),
                ("capacity", ctypes.c_int64), ("d_ngroups", ctypes.c_void_p)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("build_rows", ctypes.c_int32), ("probe_rows", ctypes.c_int32), ("lookahead", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32)]


def _load_batch(lib):
    if getattr(lib, "_batch_ready", False):
        return
    P = ctypes.POINTER
    lib.gj_batch_create.argtypes = [P(Query), ctypes.c_int32, P(BatchConfig), P(Options), P(ctypes.c_void_p),
                                    ctypes.c_void_p]
    lib.gj_batch_create.restype = ctypes.c_int32
    lib.gj_batch_launch.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.gj_batch_launch.restype = ctypes.c_int32
    lib.gj_batch_get_config.argtypes = [ctypes.c_void_p, P(BatchConfig)]
    lib.gj_batch_get_config.restype = ctypes.c_int32
    lib.gj_batch_destroy.argtypes = [ctypes.c_void_p]
    lib.gj_batch_destroy.restype = ctypes.c_int32
    lib.gj_batch_get_variants.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    lib.gj_batch_get_variants.restype = ctypes.c_int32
    lib._batch_ready = True


class BatchPlan:
    """Many join -> group-by queries run as one persistent launch (gj_batch_*).

    Each query is (rkey, rcols, skey, scols, group_key, aggs, agg_cols) with the
    conventions of join_groupby; outputs are allocated here and kept alive. Each
    query's join variant is `variant`, or with "auto" the choice of `selector`
    (None: the library default) under the given hints; queries that do not run
    the non-partitioned join in the persistent kernel run one at a time after it."""

    def __init__(self, queries, config=None, *, variant: str = "auto", selector=None,
                 match_ratio_hint: float = -1.0, zipf_hint: float = -1.0, groups_hint: int = 0):
        lib = load()
        _load_batch(lib)
        self._keep = []
        arr = (Query * max(1, len(queries)))()
        self.outputs = []
        for i, (rkey, rcols, skey, scols, gk, aggs, agg_cols) in enumerate(queries):
            q = arr[i]
            q.R = make_table(rkey, rcols)
            q.S = make_table(skey, scols)
            q.group_key = ColRef(*[int(x) for x in gk])
            q.nagg = len(aggs)
            for j, (a, ref) in enumerate(zip(aggs, agg_cols)):
                q.ops[j] = AGG[a] if isinstance(a, str) else int(a)
                q.agg_cols[j] = ColRef(*[int(x) for x in ref])
            cap = max(1, 2 * int(gk[2]) - 1) if int(gk[2]) > 0 else max(1, skey.numel())
            okeys = torch.empty(cap, dtype=torch.int64, device=rkey.device)
            oaggs = [torch.empty(cap, dtype=torch.int64, device=rkey.device) for _ in aggs]
            ng = torch.zeros(1, dtype=torch.int64, device=rkey.device)
            q.out_keys = okeys.data_ptr()
            for j, t in enumerate(oaggs):
                q.out_aggs[j] = t.data_ptr()
            q.capacity = cap
            q.d_ngroups = ng.data_ptr()
            self.outputs.append((okeys, oaggs, ng))
            self._keep.append((rkey, rcols, skey, scols))
        cfg = BatchConfig(*(config or (0, 0, 0, 0)))
        o = options(join=variant, sync=False, selector=selector, match_ratio_hint=match_ratio_hint,
                    zipf_hint=zipf_hint, groups_hint=groups_hint)
        plan = ctypes.c_void_p()
        _raise(lib.gj_batch_create(arr, len(queries), ctypes.byref(cfg), ctypes.byref(o), ctypes.byref(plan),
                                   _stream()), "gj_batch_create")
        self._plan = plan
        self._lib = lib
        self._nq = len(queries)

    def launch(self):
        _raise(self._lib.gj_batch_launch(self._plan, _stream()), "gj_batch_launch")

    def variants(self):
        """The gj_join_variant each query runs."""
        v = (ctypes.c_int32 * max(1, self._nq))()
        _raise(self._lib.gj_batch_get_variants(self._plan, ctypes.cast(v, ctypes.c_void_p)), "gj_batch_get_variants")
        return [int(v[i]) for i in range(self._nq)]

    def config(self):
        c = BatchConfig()
        _raise(self._lib.gj_batch_get_config(self._plan, ctypes.byref(c)), "gj_batch_get_config")
        return (c.build_rows, c.probe_rows, c.lookahead, c.blocks_per_sm)

    def results(self):
        """[(keys, [aggs], g)] on the host after synchronising."""
        torch.cuda.synchronize()
        out = []
        for okeys, oaggs, ng in self.outputs:
            g = int(ng.item())
            out.append((okeys[:g].cpu().numpy(), [a[:g].cpu().numpy() for a in oaggs], g))
        return out

    def close(self):
        if self._plan:
            self._lib.gj_batch_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_IN, MLP_HIDDEN, MLP_OUT, MLP_PARAMS = 12, 64, 11, 5707


def _load_mlp(lib):
    if getattr(lib, "_mlp_ready", False):
        return
    p, i32, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_float
    P = ctypes.POINTER
    lib.gj_mlp_forward.argtypes = [p, p, i32, p, p]
    lib.gj_mlp_loss_grad.argtypes = [p, p, p, p, i32, p, p, p]
    lib.gj_mlp_adam_step.argtypes = [p, p, p, p, i32, f32, f32, f32, f32, p]
    lib.gj_mlp_sgd_step.argtypes = [p, p, f32, p]
    lib.gj_mlp_select.argtypes = [p, p, i32, p, p, p]
    lib.gj_selector_set.argtypes = [p, p, p]
    lib.gj_query_features.argtypes = [P(Table), P(Table), i32, P(Options), p]
    lib.gj_heuristic_choose.argtypes = [P(Table), P(Table), i32, P(Options), P(i32), P(i32)]
    lib.gj_auto_variants.argtypes = [P(Table), P(Table), i32, p, P(Options), i32, P(i32), P(i32)]
    lib.gj_cost_params_default.argtypes = [P(CostParams)]
    lib.gj_cost_params_default.restype = None
    lib.gj_set_cost_params.argtypes = [P(CostParams)]
    lib.gj_cost_estimate.argtypes = [P(Table), P(Table), i32, p, P(Options), p, p]
    for f in ("gj_mlp_forward", "gj_mlp_loss_grad", "gj_mlp_adam_step", "gj_mlp_sgd_step", "gj_mlp_select",
              "gj_selector_set", "gj_query_features", "gj_heuristic_choose", "gj_auto_variants",
              "gj_set_cost_params", "gj_cost_estimate"):
        getattr(lib, f).restype = i32
    lib._mlp_ready = True


def _f32(t: torch.Tensor):
    assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
    return ctypes.c_void_p(t.data_ptr())


def mlp_forward(theta: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """y[b][6] of the selector network for device features x[b][12]."""
    lib = load()
    _load_mlp(lib)
    y = torch.empty((x.shape[0], MLP_OUT), dtype=torch.float32, device=x.device)
    _raise(lib.gj_mlp_forward(_f32(theta), _f32(x), x.shape[0], _f32(y), _stream()), "gj_mlp_forward")
    return y


def mlp_loss_grad(theta, x, t, mask):
    """(loss tensor[1], grad tensor[MLP_PARAMS]) of the masked squared error."""
    lib = load()
    _load_mlp(lib)
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device=x.device)
    loss = torch.empty(1, dtype=torch.float32, device=x.device)
    _raise(lib.gj_mlp_loss_grad(_f32(theta), _f32(x), _f32(t), _f32(mask), x.shape[0], _f32(grad), _f32(loss),
                                _stream()), "gj_mlp_loss_grad")
    return loss, grad


def mlp_adam_step(theta, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    lib = load()
    _load_mlp(lib)
    _raise(lib.gj_mlp_adam_step(_f32(theta), _f32(grad), _f32(m), _f32(v), step, lr, beta1, beta2, eps, _stream()),
           "gj_mlp_adam_step")


def mlp_sgd_step(theta, grad, lr):
    lib = load()
    _load_mlp(lib)
    _raise(lib.gj_mlp_sgd_step(_f32(theta), _f32(grad), lr, _stream()), "gj_mlp_sgd_step")


def mlp_select(theta, x):
    """(join variant codes, group-by variant codes) chosen by the network for each feature row."""
    lib = load()
    _load_mlp(lib)
    n = x.shape[0]
    jv = torch.empty(n, dtype=torch.int32, device=x.device)
    gv = torch.empty(n, dtype=torch.int32, device=x.device)
    _raise(lib.gj_mlp_select(_f32(theta), _f32(x), n, ctypes.c_void_p(jv.data_ptr()), ctypes.c_void_p(gv.data_ptr()),
                             _stream()), "gj_mlp_select")
    return jv, gv


def selector_set(theta_host, mean, std):
    """Install (or with theta_host None, remove) the network used by AUTO + selector=1."""
    import numpy as np
    lib = load()
    _load_mlp(lib)
    if theta_host is None:
        _raise(lib.gj_selector_set(None, None, None), "gj_selector_set")
        return
    th = np.ascontiguousarray(theta_host, dtype=np.float32)
    mu = np.ascontiguousarray(mean, dtype=np.float32)
    sd = np.ascontiguousarray(std, dtype=np.float32)
    _raise(lib.gj_selector_set(th.ctypes.data, mu.ctypes.data, sd.ctypes.data), "gj_selector_set")


def _shape_table(n: int, key_bytes: int, ncols: int, col_bytes: int = 4) -> Table:
    t = Table()
    t.key_type = I64 if key_bytes == 8 else I32
    t.ncols = ncols
    t.n = n
    for c in range(ncols):
        t.col_type[c] = I64 if col_bytes == 8 else I32
    return t


def query_features(nr, ns, key_bytes, ncols_r, ncols_s, nagg, zipf, mr, groups):
    """The 12 raw selector features of a query shape (gj_query_features)."""
    import numpy as np
    lib = load()
    _load_mlp(lib)
    R = _shape_table(nr, key_bytes, ncols_r)
    S = _shape_table(ns, key_bytes, ncols_s)
    o = options(zipf_hint=zipf, match_ratio_hint=mr, groups_hint=int(groups))
    out = np.zeros(MLP_IN, dtype=np.float32)
    _raise(lib.gj_query_features(ctypes.byref(R), ctypes.byref(S), nagg, ctypes.byref(o), out.ctypes.data),
           "gj_query_features")
    return out


def heuristic_choose(nr, ns, key_bytes, ncols_r, ncols_s, nagg, zipf, mr, groups):
    """(join variant, group-by variant) under the paper's rules (gj_heuristic_choose)."""
    lib = load()
    _load_mlp(lib)
    R = _shape_table(nr, key_bytes, ncols_r)
    S = _shape_table(ns, key_bytes, ncols_s)
    o = options(zipf_hint=zipf, match_ratio_hint=mr, groups_hint=int(groups))
    jv, gv = ctypes.c_int32(), ctypes.c_int32()
    _raise(lib.gj_heuristic_choose(ctypes.byref(R), ctypes.byref(S), nagg, ctypes.byref(o), ctypes.byref(jv),
                                   ctypes.byref(gv)), "gj_heuristic_choose")
    return jv.value, gv.value


def _ops_array(ops):
    if ops is None:
        return None, None
    arr = (ctypes.c_int32 * len(ops))(*[AGG[a] if isinstance(a, str) else int(a) for a in ops])
    return arr, ctypes.cast(arr, ctypes.c_void_p)


def auto_variants(nr, ns, key_bytes, ncols_r, ncols_s, nagg, zipf, mr, groups, *, selector=None,
                  fused: bool = False, join: str = "auto", groupby: str = "auto", ops=None):
    """(join variant, group-by variant) that AUTO requests run (gj_auto_variants):
    the join of gj_join (fused = False) or gj_join_groupby (fused = True), the
    group-by of gj_groupby over the S-shaped input with aggregates `ops` (names
    or codes; None: SUMs); host only."""
    lib = load()
    _load_mlp(lib)
    R = _shape_table(nr, key_bytes, ncols_r)
    S = _shape_table(ns, key_bytes, ncols_s)
    o = options(join=join, groupby=groupby, zipf_hint=zipf, match_ratio_hint=mr, groups_hint=int(groups),
                selector=selector)
    keep, optr = _ops_array(ops)
    jv, gv = ctypes.c_int32(), ctypes.c_int32()
    _raise(lib.gj_auto_variants(ctypes.byref(R), ctypes.byref(S), nagg, optr, ctypes.byref(o), 1 if fused else 0,
                                ctypes.byref(jv), ctypes.byref(gv)), "gj_auto_variants")
    return jv.value, gv.value


def cost_params_default() -> dict:
    """The GB300 defaults of the cost model (gj_cost_params_default)."""
    lib = load()
    _load_mlp(lib)
    p = CostParams()
    lib.gj_cost_params_default(ctypes.byref(p))
    return {f: getattr(p, f) for f, _ in CostParams._fields_ if f != "reserved"}


def set_cost_params(params=None):
    """Install cost-model parameters (a dict of gj_cost_params fields; missing ones
    keep their defaults), or with None restore the defaults."""
    lib = load()
    _load_mlp(lib)
    if params is None:
        _raise(lib.gj_set_cost_params(None), "gj_set_cost_params")
        return
    p = CostParams()
    lib.gj_cost_params_default(ctypes.byref(p))
    for k, v in params.items():
        setattr(p, k, v)
    _raise(lib.gj_set_cost_params(ctypes.byref(p)), "gj_set_cost_params")


def cost_estimate(nr, ns, key_bytes, ncols_r, ncols_s, nagg, zipf, mr, groups, *, ops=None):
    """(join costs [PHJ-TR, PHJ-UR, NPHJ, SMJ-TR, SMJ-UR], group-by costs [HGB, SGB,
    PGB, SGB-UR, PGB-UR, SGB-DE]) in bytes at B_G (gj_cost_estimate); host only.
    nr = None skips the join."""
    import numpy as np
    lib = load()
    _load_mlp(lib)
    S = _shape_table(ns, key_bytes, ncols_s)
    R = _shape_table(nr, key_bytes, ncols_r) if nr is not None else None
    o = options(zipf_hint=zipf, match_ratio_hint=mr, groups_hint=int(groups))
    keep, optr = _ops_array(ops)
    jc = np.zeros(5, dtype=np.float64)
    gc = np.zeros(6, dtype=np.float64)
    _raise(lib.gj_cost_estimate(ctypes.byref(R) if R is not None else None, ctypes.byref(S), nagg, optr,
                                ctypes.byref(o), jc.ctypes.data if R is not None else None, gc.ctypes.data),
           "gj_cost_estimate")
    return (jc if R is not None else None), gc


def profile_enable(on: bool):
    """Record CUDA events around every library kernel launch on its stream."""
    load().gj_profile_enable(1 if on else 0)


def profile_read() -> dict:
    """{kernel kind: (total ms, launches)} since the last read; synchronises the device."""
    lib = load()
    n = 32
    ms = (ctypes.c_double * n)()
    cnt = (ctypes.c_int64 * n)()
    k = lib.gj_profile_read(ms, cnt, n)
    return {lib.gj_kernel_name(i).decode(): (ms[i], cnt[i]) for i in range(k) if cnt[i]}


def kernel_launches() -> int:
    """Kernels launched by the library since it was loaded."""
    return int(load().gj_kernel_launches())


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.int32:
        return I32
    if t.dtype == torch.int64:
        return I64
    raise TypeError(f"unsupported dtype {t.dtype}: columns are int32 or int64")


def _check_dev(t: torch.Tensor, n: int):
    if not t.is_cuda:
        raise ValueError("tensors must be on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    if t.numel() != n:
        raise ValueError("all columns of a table must have the same length")


def make_table(key: torch.Tensor, cols) -> Table:
    cols = list(cols)
    if len(cols) > MAX_COLS:
        raise ValueError(f"at most {MAX_COLS} columns")
    n = key.numel()
    _check_dev(key, n)
    t = Table()
    t.key_type = _dtype_code(key)
    t.ncols = len(cols)
    t.n = n
    t.key = key.data_ptr() if n else None
    for c, col in enumerate(cols):
        _check_dev(col, n)
        t.col_type[c] = _dtype_code(col)
        t.cols[c] = col.data_ptr() if n else None
    return t


def options(join: str = "auto", groupby: str = "auto", radix_bits: int = 0, bits_per_pass: int = 0,
            sync: bool = True, zipf_hint: float = -1.0, match_ratio_hint: float = -1.0, groups_hint: int = 0,
            selector=None) -> Options:
    o = Options()
    load().gj_options_default(ctypes.byref(o))
    o.join_variant = JOIN[join]
    o.groupby_variant = GROUPBY[groupby]
    o.radix_bits = radix_bits
    o.bits_per_pass = bits_per_pass
    o.sync = 1 if sync else 0
    o.zipf_hint = zipf_hint
    o.match_ratio_hint = match_ratio_hint
    o.groups_hint = groups_hint
    if selector is not None:  # else the library's default (the cost model)
        o.selector = SELECT[selector] if isinstance(selector, str) else selector
    return o


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _raise(code: int, where: str):
    if code != 0:
        raise GjError(code, where)


def device_status() -> int:
    return load().gj_get_device_status(_stream())


def radix_partition(key: torch.Tensor, cols, bit_lo: int, bit_hi: int, transform: int = 0,
                    offsets: bool = False, bits_per_pass: int = 0, sync: bool = True):
    """Stable radix-partition of (key, cols) on bits [bit_lo, bit_hi) of d(key) (Sec. 2.3)."""
    lib = load()
    cols = list(cols)
    kin = make_table(key, cols)
    kout_t = torch.empty_like(key)
    cols_out = [torch.empty_like(c) for c in cols]
    kout = make_table(kout_t, cols_out)
    off = torch.empty((1 << (bit_hi - bit_lo)) + 1, dtype=torch.int64, device=key.device) if offsets else None
    o = options(bits_per_pass=bits_per_pass, sync=sync)
    _raise(lib.gj_radix_partition(ctypes.byref(kin), bit_lo, bit_hi, transform, ctypes.byref(kout),
                                  None if off is None else off.data_ptr(), ctypes.byref(o), _stream()),
           "gj_radix_partition")
    return kout_t, cols_out, off


def radix_partition_noalloc(key: torch.Tensor, cols, bit_lo: int, bit_hi: int, transform: int = 0,
                            offsets: bool = False, sync: bool = True, out=None):
    """radix_partition for one pass of at most 8 bits, through the entry point that
    allocates no device memory (its scratch is a fixed array in the library).
    ``out`` may pass preallocated (key, [cols]) outputs."""
    lib = load()
    if not getattr(lib, "_noalloc_ready", False):
        P = ctypes.POINTER
        lib.gj_radix_partition_noalloc.argtypes = [P(Table), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, P(Table),
                                                   ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
        lib.gj_radix_partition_noalloc.restype = ctypes.c_int32
        lib._noalloc_ready = True
    cols = list(cols)
    kin = make_table(key, cols)
    if out is None:
        out = (torch.empty_like(key), [torch.empty_like(c) for c in cols])
    kout = make_table(out[0], out[1])
    off = torch.empty((1 << (bit_hi - bit_lo)) + 1, dtype=torch.int64, device=key.device) if offsets else None
    _raise(lib.gj_radix_partition_noalloc(ctypes.byref(kin), bit_lo, bit_hi, transform, ctypes.byref(kout),
                                          None if off is None else off.data_ptr(), 1 if sync else 0, _stream()),
           "gj_radix_partition_noalloc")
    return out[0], out[1], off


def join(rkey, rcols, skey, scols, *, variant: str = "phj_tr", capacity: int | None = None,
         radix_bits: int = 0, bits_per_pass: int = 0, sync: bool = True, out=None, count=None,
         match_ratio_hint: float = -1.0, zipf_hint: float = -1.0, selector=None):
    """R join S on key (Sec. 2.2). Returns (T.key, [T.cols: R's then S's], device count tensor).

    variant: "auto", "phj_tr", "phj_ur", "nphj", "smj_tr", "smj_ur" (R.key unique), or
    "nphj_mn", "phj_mn" (many-to-many; pass a capacity that holds every pair).

    ``out`` may pass preallocated (key, cols) outputs and ``count`` a device int64[1]."""
    lib = load()
    R = make_table(rkey, rcols)
    S = make_table(skey, scols)
    if capacity is None:
        capacity = skey.numel()
    if out is None:
        tkey = torch.empty(capacity, dtype=rkey.dtype, device=rkey.device)
        tcols = [torch.empty(capacity, dtype=c.dtype, device=c.device) for c in list(rcols) + list(scols)]
    else:
        tkey, tcols = out
    T = Table()
    T.key_type = _dtype_code(tkey)
    T.ncols = len(tcols)
    T.n = capacity
    T.key = tkey.data_ptr() if capacity else None
    for c, col in enumerate(tcols):
        T.col_type[c] = _dtype_code(col)
        T.cols[c] = col.data_ptr() if capacity else None
    if count is None:
        count = torch.zeros(1, dtype=torch.int64, device=rkey.device)
    o = options(join=variant, radix_bits=radix_bits, bits_per_pass=bits_per_pass, sync=sync,
                match_ratio_hint=match_ratio_hint, zipf_hint=zipf_hint, selector=selector)
    _raise(lib.gj_join(ctypes.byref(R), ctypes.byref(S), ctypes.byref(o), ctypes.byref(T), capacity,
                       ctypes.c_void_p(count.data_ptr()), _stream()), "gj_join")
    return tkey, tcols, count


def _agg_arrays(aggs, n_out, device, capacity):
    ops = (ctypes.c_int32 * len(aggs))(*[AGG[a] if isinstance(a, str) else int(a) for a in aggs])
    outs = [torch.empty(capacity, dtype=torch.int64, device=device) for _ in aggs]
    ptrs = (ctypes.c_void_p * len(aggs))(*[t.data_ptr() if capacity else None for t in outs])
    return ops, outs, ptrs


def groupby(key, vals, aggs, agg_cols, *, variant: str = "hgb", capacity: int | None = None,
            radix_bits: int = 0, sync: bool = True, groups_hint: int = 0, zipf_hint: float = -1.0, selector=None):
    """GROUP BY key (Sec. 2.2, Alg. 1). Returns (keys, [int64 aggregate columns], device group count).

    variant: "auto", "hgb", "sgb", "pgb", "sgb_ur", "pgb_ur", "sgb_de"; selector: how "auto"
    chooses ("heuristic", "mlp", "cost" or a gj_selector_mode; None = the library default)."""
    lib = load()
    t = make_table(key, vals)
    if capacity is None:
        capacity = max(1, key.numel())
    ops, outs, ptrs = _agg_arrays(aggs, capacity, key.device, capacity)
    oc = (ctypes.c_int32 * len(aggs))(*[int(c) for c in agg_cols])
    okeys = torch.empty(capacity, dtype=key.dtype, device=key.device)
    ng = torch.zeros(1, dtype=torch.int64, device=key.device)
    o = options(groupby=variant, radix_bits=radix_bits, sync=sync, groups_hint=groups_hint, zipf_hint=zipf_hint,
                selector=selector)
    _raise(lib.gj_groupby(ctypes.byref(t), len(aggs), ops, oc, ctypes.byref(o), okeys.data_ptr(), ptrs, capacity,
                          ctypes.c_void_p(ng.data_ptr()), _stream()), "gj_groupby")
    return okeys, outs, ng


def join_groupby(rkey, rcols, skey, scols, group_key, aggs, agg_cols, *, variant: str = "auto",
                 capacity: int | None = None, radix_bits: int = 0, sync: bool = True, selector=None,
                 match_ratio_hint: float = -1.0, zipf_hint: float = -1.0, groups_hint: int = 0):
    """GROUP BY over R join S without materialising it. group_key / agg_cols are
    (side, col, modulus) triples (side 0 = R, 1 = S; col -1 = join key); selector and
    hints as for join / groupby."""
    lib = load()
    R = make_table(rkey, rcols)
    S = make_table(skey, scols)
    if capacity is None:
        capacity = max(1, skey.numel())
    ops, outs, ptrs = _agg_arrays(aggs, capacity, rkey.device, capacity)
    refs = (ColRef * len(aggs))(*[ColRef(int(s), int(c), int(m)) for s, c, m in agg_cols])
    gk = ColRef(*[int(x) for x in group_key])
    okeys = torch.empty(capacity, dtype=torch.int64, device=rkey.device)
    ng = torch.zeros(1, dtype=torch.int64, device=rkey.device)
    o = options(join=variant, radix_bits=radix_bits, sync=sync, selector=selector, match_ratio_hint=match_ratio_hint,
                zipf_hint=zipf_hint, groups_hint=groups_hint)
    _raise(lib.gj_join_groupby(ctypes.byref(R), ctypes.byref(S), gk, len(aggs), ops, refs, ctypes.byref(o),
                               okeys.data_ptr(), ptrs, capacity, ctypes.c_void_p(ng.data_ptr()), _stream()),
           "gj_join_groupby")
    return okeys, outs, ng
