"""Thin ctypes binding of the C ABI in include/legcheb.h.

Argument marshalling only: every function here forwards to the function of
the same name in liblegcheb.so and raises LegChebError on a non-zero status.
There is no fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "liblegcheb.so"

LC_L2C, LC_C2L = 0, 1
#: largest n that lc_direct_static accepts (LC_STATIC_MAX_N in include/legcheb.h)
LC_STATIC_MAX_N = 16384
#: largest n of a plan with values at Chebyshev points (LC_VALUES_MAX_N)
LC_VALUES_MAX_N = 4194304
#: largest n that is not a power of two of a plan with values at Chebyshev points
LC_VALUES_MAX_N_ANY = 2097152
#: largest Gegenbauer parameter a of a plan (LC_GEGENBAUER_MAX_ALPHA)
LC_GEGENBAUER_MAX_ALPHA = 2.0
LC_F64, LC_F64_SPLIT, LC_F32, LC_F64_DF = 0, 1, 2, 3
STATUS_NAMES = {
    0: "LC_OK", 1: "LC_ERR_INVALID_ARG", 2: "LC_ERR_WORKSPACE_TOO_SMALL", 3: "LC_ERR_CUDA",
    4: "LC_ERR_DEVICE_TIMEOUT", 5: "LC_ERR_UNSUPPORTED", 6: "LC_ERR_HOST_ALLOC",
}

#: every symbol declared in include/legcheb.h
EXPORTED = (
    "lc_plan_options_default", "lc_plan_workspace_size", "lc_plan_workspace_size_ex",
    "lc_plan_create", "lc_plan_create_ex", "lc_plan_workspace_size_ragged", "lc_plan_create_ragged",
    "lc_execute", "lc_adjoint", "lc_destroy", "lc_status_string", "lc_plan_info", "lc_plan_table",
    "lc_plan_launches", "lc_plan_set_timing", "lc_plan_get_timing", "lc_plan_check", "lc_direct_static",
    "lc_plan_set_config", "lc_plan_autotune", "lc_execute_ex", "lc_adjoint_ex", "lc_plan_set_band",
    "lc_plan_set_split_schedule",
)


class LegChebError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s: %s" % (where, STATUS_NAMES.get(status, "status %d" % status)))


class PlanOptions(ctypes.Structure):
    _fields_ = [("s_hat", ctypes.c_int32), ("fixed_s", ctypes.c_int32), ("slices", ctypes.c_int32),
                ("debug_flags", ctypes.c_int32), ("values", ctypes.c_int32), ("nodal", ctypes.c_int32), ("fp64_plan", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1),
                ("alpha", ctypes.c_double)]


_lib = None


def library_path() -> Path:
    return _LIB_PATH


def load(path: Path | None = None):
    """Load liblegcheb.so (built by paper_2411_00033_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else _LIB_PATH
    if not p.exists():
        raise ImportError(
            "liblegcheb.so is not built (%s); run `python -c 'import __graft_entry__ as g; g.build()'`" % p)
    lib = ctypes.CDLL(str(p))
    i32, i64, sz, vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p
    p64, pi32, psz = ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(sz)
    popt = ctypes.POINTER(PlanOptions)
    sig = {
        "lc_plan_options_default": [popt],
        "lc_plan_workspace_size": [i64, ctypes.c_int, i64, ctypes.c_int, psz],
        "lc_plan_workspace_size_ex": [i64, ctypes.c_int, i64, ctypes.c_int, popt, psz],
        "lc_plan_create": [ctypes.POINTER(vp), i64, ctypes.c_int, i64, ctypes.c_int, vp, sz, vp],
        "lc_plan_create_ex": [ctypes.POINTER(vp), i64, ctypes.c_int, i64, ctypes.c_int, popt, vp, sz, vp],
        "lc_plan_workspace_size_ragged": [p64, i64, ctypes.c_int, ctypes.c_int, popt, psz],
        "lc_plan_create_ragged": [ctypes.POINTER(vp), p64, i64, ctypes.c_int, ctypes.c_int, popt, vp, sz, vp],
        "lc_execute": [vp, vp, vp, i64, i64, i64, i64, vp],
        "lc_adjoint": [vp, vp, vp, i64, i64, i64, i64, vp],
        "lc_execute_ex": [vp, vp, vp, i64, i64, i64, i64, i64, i64, i64, vp],
        "lc_adjoint_ex": [vp, vp, vp, i64, i64, i64, i64, i64, i64, i64, vp],
        "lc_destroy": [vp],
        "lc_plan_info": [vp, p64, p64, pi32, pi32, pi32, p64, p64],
        "lc_plan_table": [vp, i32, ctypes.POINTER(ctypes.c_double), i64, p64, vp],
        "lc_plan_launches": [vp, pi32],
        "lc_plan_set_timing": [vp, i32],
        "lc_plan_check": [vp, vp],
        "lc_plan_set_config": [vp, i32, i32],
        "lc_plan_set_band": [vp, i32, i32],
        "lc_plan_set_split_schedule": [vp, i32],
        "lc_plan_autotune": [vp, vp, vp, i64, i64, i64, i64, vp, pi32, pi32, ctypes.POINTER(ctypes.c_float)],
        "lc_plan_get_timing": [vp, i32, ctypes.POINTER(ctypes.c_float), pi32, i32, pi32],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.lc_status_string.argtypes = [ctypes.c_int]
    lib.lc_status_string.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        raise LegChebError(status, where)


def lc_status_string(status: int) -> str:
    return load().lc_status_string(status).decode()


def lc_plan_options_default() -> PlanOptions:
    o = PlanOptions()
    _check(load().lc_plan_options_default(ctypes.byref(o)), "lc_plan_options_default")
    return o


def lc_plan_workspace_size(n, direction, batch, dtype, options: PlanOptions | None = None) -> int:
    b = ctypes.c_size_t()
    opt = ctypes.byref(options) if options is not None else None
    _check(load().lc_plan_workspace_size_ex(n, direction, batch, dtype, opt, ctypes.byref(b)),
           "lc_plan_workspace_size")
    return b.value


def lc_plan_create(n, direction, batch, dtype, workspace_ptr, nbytes, stream_ptr,
                   options: PlanOptions | None = None) -> int:
    h = ctypes.c_void_p()
    opt = ctypes.byref(options) if options is not None else None
    _check(load().lc_plan_create_ex(ctypes.byref(h), n, direction, batch, dtype, opt,
                                    ctypes.c_void_p(workspace_ptr), nbytes, ctypes.c_void_p(stream_ptr)),
           "lc_plan_create")
    return h.value


def _i64_array(values):
    arr = (ctypes.c_int64 * len(values))(*[int(v) for v in values])
    return arr


def lc_plan_workspace_size_ragged(lengths, direction, dtype, options: PlanOptions | None = None) -> int:
    b = ctypes.c_size_t()
    arr = _i64_array(lengths)
    opt = ctypes.byref(options) if options is not None else None
    _check(load().lc_plan_workspace_size_ragged(arr, len(lengths), direction, dtype, opt, ctypes.byref(b)),
           "lc_plan_workspace_size_ragged")
    return b.value


def lc_plan_create_ragged(lengths, direction, dtype, workspace_ptr, nbytes, stream_ptr,
                          options: PlanOptions | None = None) -> int:
    h = ctypes.c_void_p()
    arr = _i64_array(lengths)
    opt = ctypes.byref(options) if options is not None else None
    _check(load().lc_plan_create_ragged(ctypes.byref(h), arr, len(lengths), direction, dtype, opt,
                                        ctypes.c_void_p(workspace_ptr), nbytes, ctypes.c_void_p(stream_ptr)),
           "lc_plan_create_ragged")
    return h.value


def lc_execute(plan, in_ptr, out_ptr, ib, ie, ob, oe, stream_ptr):
    _check(load().lc_execute(ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
                             ib, ie, ob, oe, ctypes.c_void_p(stream_ptr)), "lc_execute")


def lc_adjoint(plan, in_ptr, out_ptr, ib, ie, ob, oe, stream_ptr):
    _check(load().lc_adjoint(ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
                             ib, ie, ob, oe, ctypes.c_void_p(stream_ptr)), "lc_adjoint")


def lc_execute_ex(plan, in_ptr, out_ptr, ib, ie, ob, oe, inner, iob, oob, stream_ptr):
    _check(load().lc_execute_ex(ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
                                ib, ie, ob, oe, inner, iob, oob, ctypes.c_void_p(stream_ptr)), "lc_execute_ex")


def lc_adjoint_ex(plan, in_ptr, out_ptr, ib, ie, ob, oe, inner, iob, oob, stream_ptr):
    _check(load().lc_adjoint_ex(ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr),
                                ib, ie, ob, oe, inner, iob, oob, ctypes.c_void_p(stream_ptr)), "lc_adjoint_ex")


def lc_destroy(plan):
    _check(load().lc_destroy(ctypes.c_void_p(plan)), "lc_destroy")


def lc_plan_info(plan) -> dict:
    n, N, nc, batch = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    L, s, M = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().lc_plan_info(ctypes.c_void_p(plan), ctypes.byref(n), ctypes.byref(N), ctypes.byref(L),
                               ctypes.byref(s), ctypes.byref(M), ctypes.byref(nc), ctypes.byref(batch)),
           "lc_plan_info")
    return dict(n=n.value, N=N.value, L=L.value, s=s.value, M=M.value, n_c=nc.value, batch=batch.value)


def lc_plan_table(plan, which: int, count: int, stream_ptr):
    import numpy as np
    buf = np.empty(max(count, 1), np.float64)
    copied = ctypes.c_int64()
    _check(load().lc_plan_table(ctypes.c_void_p(plan), which, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                count, ctypes.byref(copied), ctypes.c_void_p(stream_ptr)), "lc_plan_table")
    return buf[:copied.value].copy()


def lc_plan_launches(plan) -> int:
    v = ctypes.c_int32()
    _check(load().lc_plan_launches(ctypes.c_void_p(plan), ctypes.byref(v)), "lc_plan_launches")
    return v.value


def lc_plan_check(plan, stream_ptr):
    """Raise LegChebError(LC_ERR_DEVICE_TIMEOUT) if a bounded device wait ran out."""
    _check(load().lc_plan_check(ctypes.c_void_p(plan), ctypes.c_void_p(stream_ptr)), "lc_plan_check")


def lc_plan_set_timing(plan, slots: int):
    _check(load().lc_plan_set_timing(ctypes.c_void_p(plan), slots), "lc_plan_set_timing")


def lc_plan_get_timing(plan, slot: int, capacity: int = 256):
    """[(kind, ms)] for the kernels of the execution recorded in `slot`."""
    ms = (ctypes.c_float * capacity)()
    kinds = (ctypes.c_int32 * capacity)()
    count = ctypes.c_int32()
    _check(load().lc_plan_get_timing(ctypes.c_void_p(plan), slot, ms, kinds, capacity, ctypes.byref(count)),
           "lc_plan_get_timing")
    return [(int(kinds[i]), float(ms[i])) for i in range(min(count.value, capacity))]


def lc_direct_static(direction, n, batch, in_ptr, out_ptr, ib, ie, ob, oe, stream_ptr):
    """Direct transform whose only scratch is a static device array (no allocation)."""
    lib = load()
    f = lib.lc_direct_static
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    _check(f(direction, n, batch, ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), ib, ie, ob, oe,
             ctypes.c_void_p(stream_ptr)), "lc_direct_static")


def lc_plan_set_config(plan, leaf_depth: int, chunk_depth: int):
    _check(load().lc_plan_set_config(ctypes.c_void_p(plan), leaf_depth, chunk_depth), "lc_plan_set_config")


def lc_plan_set_band(plan, ctas: int, after_leaf: int):
    _check(load().lc_plan_set_band(ctypes.c_void_p(plan), ctas, after_leaf), "lc_plan_set_band")


def lc_plan_set_split_schedule(plan, persistent: int):
    _check(load().lc_plan_set_split_schedule(ctypes.c_void_p(plan), persistent), "lc_plan_set_split_schedule")


def lc_plan_autotune(plan, in_ptr, out_ptr, ib, ie, ob, oe, stream_ptr):
    """Time the candidate chunk geometries, keep the fastest: returns (leaf_depth, chunk_depth, ms)."""
    a, b, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_float()
    _check(load().lc_plan_autotune(ctypes.c_void_p(plan), ctypes.c_void_p(in_ptr), ctypes.c_void_p(out_ptr), ib, ie,
                                   ob, oe, ctypes.c_void_p(stream_ptr), ctypes.byref(a), ctypes.byref(b),
                                   ctypes.byref(ms)), "lc_plan_autotune")
    return a.value, b.value, ms.value
