"""Thin ctypes binding of libdd.so: the C ABI of include/dd.h, same names.

Argument marshalling only: every step of the path runs in the library's
CUDA kernels.  Buffers may be torch tensors (device or host) or numpy arrays
(host); their data pointers are passed through unchanged.  If the library is
missing this module raises ImportError -- there is no fallback.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libdd.so")

DD_OK, DD_EINVAL, DD_ENOMEM, DD_ECUDA, DD_ESTATE, DD_ENOTCONV, DD_ETIMEOUT, DD_EBUDGET = 0, -1, -2, -3, -4, -5, -6, -7
DD_F_KL, DD_F_TV, DD_F_KLT = 1, 2, 4
DD_PREC_FP32, DD_PREC_BF16X3, DD_PREC_SPARSE, DD_PREC_SPARSE_MERGED = 0, 1, 2, 3
DD_FAST_LOG_SPREAD, DD_EXACT_BELOW, DD_TILE_EXACT_BELOW = 5.0e-7, 0.05, 0.25
DD_DIV_CHI2, DD_DIV_HELLINGER, DD_DIV_POWER, DD_DIV_ALPHA, DD_DIV_KL_REVERSE = 1, 2, 3, 4, 5
DD_TRACE_OK, DD_TRACE_STUCK, DD_TRACE_STEP_LIMIT, DD_TRACE_TRUNCATED = 0, 1, 2, 3

STATUS_NAMES = {0: "DD_OK", -1: "DD_EINVAL", -2: "DD_ENOMEM", -3: "DD_ECUDA", -4: "DD_ESTATE",
                -5: "DD_ENOTCONV", -6: "DD_ETIMEOUT", -7: "DD_EBUDGET"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libdd.so is not built ({LIB_PATH}); run paper_1708_02845_gb300.build.build()")

lib = ctypes.CDLL(LIB_PATH)

_p = ctypes.c_void_p
_i32 = ctypes.c_int32
_i64 = ctypes.c_int64
_u32 = ctypes.c_uint32
_f64 = ctypes.c_double

_SIGS = {
    "dd_version": (_i32, []),
    "dd_create": (_i32, [ctypes.POINTER(_p), _i32, _p]),
    "dd_set_stream": (_i32, [_p, _p]),
    "dd_destroy": (None, [_p]),
    "dd_last_error": (ctypes.c_char_p, [_p]),
    "dd_sync": (_i32, [_p]),
    "dd_check_mesh": (_i32, [_p, _i64, _p, _i64, _p, _p, _i32, _p, ctypes.c_char_p, _i32]),
    "dd_load_mesh": (_i32, [_p, _p, _i64, _p, _i64, _p, _p, _i32, ctypes.POINTER(_i32)]),
    "dd_unload_mesh": (_i32, [_p, _i32]),
    "dd_mesh_info": (_i32, [_p, _i32, _p]),
    "dd_poisson_kernel": (_i32, [_p, _i32, _f64, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_f64)]),
    "dd_set_poisson_kernel": (_i32, [_p, _i32, _p]),
    "dd_get_poisson_kernel": (_i32, [_p, _i32, _p]),
    "dd_log_poisson_kernel": (_i32, [_p, _i32, _f64, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_f64)]),
    "dd_get_log_poisson_kernel": (_i32, [_p, _i32, _p]),
    "dd_sparsify": (_i32, [_p, _i32, _f64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "dd_distance": (_i32, [_p, _i32, _p, _i32, _u32, _i32, _p]),
    "dd_divergence": (_i32, [_p, _i32, _p, _i32, _i32, _f64, _p]),
    "dd_local_minima": (_i32, [_p, _i32, _p, _p, _i32, _p, _p]),
    "dd_trace_edges": (_i32, [_p, _i32, _p, _p, _i32, _p, _i32, _i32, _p, _p, _p]),
    "dd_trace": (_i32, [_p, _i32, _i32, _u32, _p, _i32, _i32, _p, _p, _p]),
    "dd_trace_fields": (_i32, [_p, _i32, _p, _p, _i32, _p, _i32, _i32, _p, _p, _p]),
    "dd_query": (_i32, [_p, _i32, _p, _i32, _p, _i32, _u32, _i32, _u32, _i32, _p, _p, _p, _p]),
    "dd_distance_noalloc": (_i32, [_p, _i64, _i64, _p, _i32, _u32, _p, _p]),
    "dd_query_batch": (_i32, [_p, _i32, _p, _p, _p, _p, _i32, _u32, _u32, _i32, _p, _p, _p, _p]),
    "dd_tuning_table": (_i32, [ctypes.c_char_p, _i32]),
    "dd_kernel_timing": (_i32, [_p, _i32, ctypes.c_char_p, _i32]),
    "dd_load_latency": (_i32, [_p, _i64, _i32, ctypes.POINTER(ctypes.c_double)]),
    "dd_check_fast_log": (_i32, [ctypes.POINTER(ctypes.c_double)]),
    "dd_multigrid_check": (_i32, [_p, _p, _p, _i64, _p, _p, _f64, _i32, _p, _p]),
    "dd_server_create": (_i32, [_p, _i64, _i32, _i32, _i32, ctypes.POINTER(_p)]),
    "dd_server_submit": (_i32, [_p, _i64, _i32, _i32, _p, _i32]),
    "dd_server_poll": (_i32, [_p, _i32, _p, _p, _p]),
    "dd_server_take": (_i32, [_p, _i64, _p, _p, _p]),
    "dd_server_wait_idle": (_i32, [_p, _f64]),
    "dd_server_destroy": (None, [_p]),
}

for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class DDError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def ptr(x):
    """Data pointer of a torch tensor, numpy array or None (must be contiguous)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check(ctx, st):
    if st != DD_OK:
        msg = lib.dd_last_error(ctx).decode() if ctx else ""
        raise DDError(st, msg)


def _host_i32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.int32))


# ---- same names as the C ABI -------------------------------------------------

def dd_version() -> int:
    return lib.dd_version()


def dd_create(device: int = 0, stream: int = 0):
    h = _p()
    st = lib.dd_create(ctypes.byref(h), device, stream or None)
    if st != DD_OK:
        raise DDError(st, f"dd_create(device={device}) failed")
    return h


def dd_set_stream(ctx, stream: int):
    _check(ctx, lib.dd_set_stream(ctx, stream or None))


def dd_destroy(ctx):
    lib.dd_destroy(ctx)


def dd_last_error(ctx) -> str:
    return lib.dd_last_error(ctx).decode()


def dd_sync(ctx):
    _check(ctx, lib.dd_sync(ctx))


def dd_check_mesh(xy, tri, loop_idx, loop_off):
    """Host-only validation; returns (n_v, k, m, n_edges) or raises DDError."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = _host_i32(tri)
    loop_idx = _host_i32(loop_idx)
    loop_off = np.ascontiguousarray(loop_off, dtype=np.int64)
    info = np.zeros(4, dtype=np.int64)
    msg = ctypes.create_string_buffer(512)
    st = lib.dd_check_mesh(ptr(xy), xy.shape[0], ptr(tri), tri.shape[0], ptr(loop_idx), ptr(loop_off),
                           len(loop_off) - 1, ptr(info), msg, 512)
    if st != DD_OK:
        raise DDError(st, msg.value.decode())
    return tuple(int(v) for v in info)


def dd_load_mesh(ctx, xy, tri, loop_idx, loop_off) -> int:
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = _host_i32(tri)
    loop_idx = _host_i32(loop_idx)
    loop_off = np.ascontiguousarray(loop_off, dtype=np.int64)
    mid = _i32()
    _check(ctx, lib.dd_load_mesh(ctx, ptr(xy), xy.shape[0], ptr(tri), tri.shape[0], ptr(loop_idx), ptr(loop_off),
                                 len(loop_off) - 1, ctypes.byref(mid)))
    return mid.value


def dd_unload_mesh(ctx, mesh: int):
    _check(ctx, lib.dd_unload_mesh(ctx, mesh))


def dd_mesh_info(ctx, mesh: int) -> dict:
    info = np.zeros(7, dtype=np.int64)
    _check(ctx, lib.dd_mesh_info(ctx, mesh, ptr(info)))
    keys = ("n_v", "n_t", "k", "m", "k_pad", "has_poisson_kernel", "device_bytes")
    return {k: int(v) for k, v in zip(keys, info)}


def dd_poisson_kernel(ctx, mesh: int, rtol: float = 1e-15, max_iter: int = 20000, allow_notconv=False):
    iters = _i32()
    resid = _f64()
    st = lib.dd_poisson_kernel(ctx, mesh, rtol, max_iter, ctypes.byref(iters), ctypes.byref(resid))
    if not (allow_notconv and st == DD_ENOTCONV):
        _check(ctx, st)
    return iters.value, resid.value


def dd_set_poisson_kernel(ctx, mesh: int, P):
    P = np.ascontiguousarray(P, dtype=np.float64)
    _check(ctx, lib.dd_set_poisson_kernel(ctx, mesh, ptr(P)))


def dd_get_poisson_kernel(ctx, mesh: int, out):
    _check(ctx, lib.dd_get_poisson_kernel(ctx, mesh, ptr(out)))
    return out


def dd_log_poisson_kernel(ctx, mesh: int, tol: float = 1e-14, max_sweeps: int = 200000, allow_notconv=False):
    """Refine P to full relative precision in every entry and store log2 P; returns (sweeps, last change)."""
    sweeps = _i32()
    change = _f64()
    st = lib.dd_log_poisson_kernel(ctx, mesh, tol, max_sweeps, ctypes.byref(sweeps), ctypes.byref(change))
    if not (allow_notconv and st == DD_ENOTCONV):
        _check(ctx, st)
    return sweeps.value, change.value


def dd_get_log_poisson_kernel(ctx, mesh: int, out):
    _check(ctx, lib.dd_get_log_poisson_kernel(ctx, mesh, ptr(out)))
    return out


def dd_sparsify(ctx, mesh: int, theta: float = -1.0):
    """Sparse copy of P for DD_PREC_SPARSE(_MERGED); returns (kept entries, bytes of the CSR copy)."""
    kept, nbytes = _i64(0), _i64(0)
    _check(ctx, lib.dd_sparsify(ctx, mesh, float(theta), ctypes.byref(kept), ctypes.byref(nbytes)))
    return kept.value, nbytes.value


def dd_distance(ctx, mesh: int, targets, f_mask: int, prec: int, out):
    t = _host_i32(targets)
    _check(ctx, lib.dd_distance(ctx, mesh, ptr(t), len(t), f_mask, prec, ptr(out)))
    return out


def dd_divergence(ctx, mesh: int, targets, family: int, param: float, out):
    """Other f-divergence fields (DD_DIV_*), out [T][n_v] on the device or host."""
    t = _host_i32(targets)
    _check(ctx, lib.dd_divergence(ctx, mesh, ptr(t), len(t), int(family), float(param), ptr(out)))
    return out


def dd_local_minima(ctx, mesh: int, fields, targets, flags=None):
    """Spurious local minima of device fields [T][n_v]; returns counts [T]."""
    t = _host_i32(targets)
    counts = np.zeros(len(t), dtype=np.int32)
    _check(ctx, lib.dd_local_minima(ctx, mesh, ptr(fields), ptr(t), len(t), counts.ctypes.data,
                                    ptr(flags) if flags is not None else None))
    return counts


def dd_trace_edges(ctx, mesh: int, fields, targets, sources, max_pts: int, out_xy, out_len, out_status):
    t = _host_i32(targets)
    s = np.ascontiguousarray(_host_i32(sources).reshape(len(t), -1))
    _check(ctx, lib.dd_trace_edges(ctx, mesh, ptr(fields), ptr(t), len(t), ptr(s), s.shape[1], max_pts,
                                   ptr(out_xy), ptr(out_len), ptr(out_status)))


def dd_trace(ctx, mesh: int, target: int, f: int, sources, max_pts: int, out_xy, out_len, out_status):
    s = _host_i32(sources)
    _check(ctx, lib.dd_trace(ctx, mesh, int(target), f, ptr(s), len(s), max_pts, ptr(out_xy), ptr(out_len),
                             ptr(out_status)))


def dd_trace_fields(ctx, mesh: int, fields, targets, sources, max_pts: int, out_xy, out_len, out_status):
    t = _host_i32(targets)
    s = _host_i32(sources).reshape(len(t), -1)
    s = np.ascontiguousarray(s)
    _check(ctx, lib.dd_trace_fields(ctx, mesh, ptr(fields), ptr(t), len(t), ptr(s), s.shape[1], max_pts,
                                    ptr(out_xy), ptr(out_len), ptr(out_status)))


def dd_query(ctx, mesh: int, targets, sources, f_mask: int, prec: int, trace_f: int, max_pts: int,
             out_fields, out_xy, out_len, out_status):
    t = _host_i32(targets)
    s = np.ascontiguousarray(_host_i32(sources).reshape(len(t), -1))
    _check(ctx, lib.dd_query(ctx, mesh, ptr(t), len(t), ptr(s), s.shape[1], f_mask, prec, trace_f, max_pts,
                             ptr(out_fields), ptr(out_xy), ptr(out_len), ptr(out_status)))


def dd_distance_noalloc(P, n_v: int, k_pad: int, targets, T: int, f_mask: int, out, stream: int = 0):
    """Fields without device allocation: P, targets and out are device buffers."""
    st = lib.dd_distance_noalloc(ptr(P), n_v, k_pad, ptr(targets), T, f_mask, ptr(out), stream or None)
    if st != DD_OK:
        raise DDError(st, "dd_distance_noalloc failed")
    return out


def dd_query_batch(ctx, mesh_ids, T_per, targets, sources, S: int, f_mask: int, trace_f: int, max_pts: int,
                   out_fields, out_xy=None, out_len=None, out_status=None):
    """Several meshes in one pass; targets/sources concatenated item after item."""
    mids = _host_i32(mesh_ids)
    tp = _host_i32(T_per)
    t = _host_i32(targets)
    s = _host_i32(sources) if S > 0 else np.zeros(1, np.int32)
    _check(ctx, lib.dd_query_batch(ctx, len(mids), ptr(mids), ptr(tp), ptr(t), ptr(s), S, f_mask, trace_f, max_pts,
                                   ptr(out_fields), ptr(out_xy), ptr(out_len), ptr(out_status)))


def dd_check_fast_log() -> float:
    """Spread (max - min) of the hardware base-2 log's error over [1, 2)."""
    v = ctypes.c_double()
    st = lib.dd_check_fast_log(ctypes.byref(v))
    if st != DD_OK:
        raise DDError(st, "dd_check_fast_log failed")
    return v.value


def dd_multigrid_check(a_off, a_col, a_val, b, rtol: float = 1e-12, max_iter: int = 200):
    """Host-only multigrid-preconditioned CG on the CSR matrix (no GPU).
    Returns (x, iterations, levels)."""
    a_off = np.ascontiguousarray(a_off, dtype=np.int64)
    a_col = np.ascontiguousarray(a_col, dtype=np.int32)
    a_val = np.ascontiguousarray(a_val, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = len(a_off) - 1
    x = np.zeros(n, dtype=np.float64)
    it, lv = ctypes.c_int32(), ctypes.c_int32()
    st = lib.dd_multigrid_check(a_off.ctypes.data, a_col.ctypes.data, a_val.ctypes.data, n, b.ctypes.data,
                                x.ctypes.data, float(rtol), int(max_iter), ctypes.byref(it), ctypes.byref(lv))
    if st != DD_OK:
        raise DDError(st, "dd_multigrid_check failed")
    return x, it.value, lv.value


def dd_tuning_table() -> str:
    n = lib.dd_tuning_table(None, 0)
    buf = ctypes.create_string_buffer(max(n, 0) + 1)
    lib.dd_tuning_table(buf, len(buf))
    return buf.value.decode()


def dd_server_create(ctx, budget_bytes: int, n_slots: int = 3, max_batch: int = 64, max_pts: int = 2048):
    h = _p()
    st = lib.dd_server_create(ctx, int(budget_bytes), n_slots, max_batch, max_pts, ctypes.byref(h))
    if st != DD_OK:
        raise DDError(st, "dd_server_create failed")
    return h


def dd_server_submit(sv, query_id: int, mesh: int, target: int, sources) -> int:
    """Returns the status (DD_OK, or DD_EBUDGET for a query that can never fit); raises on bad arguments."""
    s = _host_i32(sources)
    st = lib.dd_server_submit(sv, int(query_id), int(mesh), int(target), ptr(s), len(s))
    if st not in (DD_OK, DD_EBUDGET):
        raise DDError(st, "dd_server_submit failed")
    return st


def dd_server_poll(sv, max_n: int = 4096):
    ids = np.zeros(max_n, np.int64)
    sts = np.zeros(max_n, np.int32)
    lat = np.zeros(max_n, np.float64)
    n = lib.dd_server_poll(sv, max_n, ptr(ids), ptr(sts), ptr(lat))
    return ids[:n], sts[:n], lat[:n]


def dd_server_take(sv, query_id: int, S: int, max_pts: int):
    xy = np.zeros((S, max_pts, 2), np.float32)
    ln = np.zeros(S, np.int32)
    st = np.zeros(S, np.int32)
    code = lib.dd_server_take(sv, int(query_id), ptr(xy), ptr(ln), ptr(st))
    if code != DD_OK:
        raise DDError(code, "dd_server_take failed")
    return xy, ln, st


def dd_server_wait_idle(sv, timeout_s: float = 60.0):
    st = lib.dd_server_wait_idle(sv, float(timeout_s))
    if st != DD_OK:
        raise DDError(st, "dd_server_wait_idle timed out")


def dd_server_destroy(sv):
    lib.dd_server_destroy(sv)


def dd_load_latency(ctx, nbytes: int, steps: int) -> float:
    """ns per dependent global load along a random cycle through nbytes."""
    ns = ctypes.c_double(0.0)
    _check(ctx, lib.dd_load_latency(ctx, int(nbytes), int(steps), ctypes.byref(ns)))
    return ns.value


def dd_kernel_timing(ctx, mode: int) -> dict:
    """mode 1: enable/reset, 2: read, 0: read and disable; returns
    {kernel name: (launches, total ms)} of what was read."""
    if mode == 1:
        st = lib.dd_kernel_timing(ctx, 1, None, 0)
        if st < 0:
            raise DDError(st, "dd_kernel_timing")
        return {}
    n = lib.dd_kernel_timing(ctx, 2, None, 0)
    if n < 0:
        raise DDError(n, "dd_kernel_timing")
    buf = ctypes.create_string_buffer(n + 1)
    lib.dd_kernel_timing(ctx, 2, buf, len(buf))
    if mode == 0:
        lib.dd_kernel_timing(ctx, 0, None, 0)
    out = {}
    for line in buf.value.decode().splitlines():
        name, cnt, ms = line.rsplit(" ", 2)
        out[name] = (int(cnt), float(ms))
    return out
