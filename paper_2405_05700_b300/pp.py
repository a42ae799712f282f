"""Python binding of the C ABI in ``include/pp.h`` (ctypes, marshalling only).

Every ``pp_*`` function here has the name and argument order of the C entry
point it calls; numpy arrays are passed as host pointers and torch CUDA
tensors (or raw integers) as device pointers.  All arithmetic runs in the
CUDA library ``libpp.so``; if that library is missing this module raises on
import -- there is no CPU fallback.

``Propagator`` wraps a context with the same calls on numpy / torch inputs.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import workloads

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpp.so")

PP_OK, PP_EINVAL, PP_ENOTLOADED, PP_EBUDGET = 0, -1, -2, -3
PP_ETIMEDOUT, PP_ECUDA, PP_EDEVICE, PP_ENOMEM, PP_ENODEV = -4, -5, -6, -7, -8
PP_OUT_ABSORBED, PP_OUT_ESCAPED, PP_OUT_TRUNCATED = -1, -2, -3


class pp_config(C.Structure):
    _fields_ = [
        ("device", C.c_int32), ("max_steps", C.c_uint32), ("seed", C.c_uint64),
        ("world_margin_m", C.c_float),
        ("depth_of_z0_m", C.c_float), ("scatter_coeff_is_effective", C.c_int32),
        ("reserved", C.c_int32), ("stream", C.c_void_p),
    ]


class pp_source(C.Structure):
    _fields_ = [
        ("x", C.c_float), ("y", C.c_float), ("z", C.c_float),
        ("dx", C.c_float), ("dy", C.c_float), ("dz", C.c_float),
        ("length", C.c_float), ("type", C.c_uint32), ("n_photons", C.c_uint64),
    ]


assert C.sizeof(pp_source) == workloads.SOURCE_DTYPE.itemsize == 40

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_2405_05700_b300.build` (needs nvcc)")

_lib = C.CDLL(LIB_PATH)

_vp, _i32, _i64, _u64 = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64
_SIGS = {
    "pp_config_default": [_vp],
    "pp_create": [_vp, _vp],
    "pp_destroy": [_vp],
    "pp_load_geometry": [_vp, _vp, _vp, _i32, C.c_float],
    "pp_load_ice": [_vp, _vp, _vp, _i32, C.c_float, C.c_float, C.c_float],
    "pp_propagate": [_vp, _u64, _vp, _i64, _vp, _vp],
    "pp_propagate_batch": [_vp, _i32, _vp, _vp, _vp, _vp, _vp],
    "pp_propagate_batch_async": [_vp, _i32, _vp, _vp, _vp, _i64, _vp, _vp, _vp],
    "pp_propagate_plain_async": [_vp, _i32, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "pp_propagate_noalloc": [_vp, _u64, _vp, _i64, _vp, _vp, _vp],
    "pp_propagate_records_async": [_vp, _i32, _vp, _vp, _vp, _i64, _vp, _vp, C.c_float, _vp, _u64,
                                   _vp, _vp],
    "pp_propagate_range_async": [_vp, _u64, _vp, _i64, _u64, _u64, _i32, _vp, _vp, _vp],
    "pp_sync": [_vp, _vp],
    "pp_set_launch": [_vp, _i32, _i32, _i32, _i32],
    "pp_autotune_batch": [_vp, _i32, _vp, _vp, _vp, _i64, _vp, _vp, _vp, _i32, _vp, _vp],
    "pp_get_launch": [_vp, _vp, _vp, _vp, _vp, _vp],
    "pp_get_world": [_vp, _vp],
    "pp_set_kernel_timing": [_vp, _i32],
    "pp_set_graphs": [_vp, _i32],
    "pp_get_path_stats": [_vp, _vp],
    "pp_get_memory": [_vp, _vp, _vp],
    "pp_get_kernel_time": [_vp, _vp, _vp, _vp],
    "pp_server_config_default": [_vp],
    "pp_server_create": [_vp, _vp, _vp],
    "pp_server_destroy": [_vp],
    "pp_submit": [_vp, _u64, _vp, _i64, _vp],
    "pp_collect": [_vp, _u64, _vp, _vp, _i32],
    "pp_server_stats": [_vp, _vp],
    "pp_mlp_create": [_vp, _i32, _i64, _vp],
    "pp_mlp_destroy": [_vp],
    "pp_mlp_set_params": [_vp, _vp, _i64],
    "pp_mlp_get_params": [_vp, _vp, _i64],
    "pp_mlp_get_state": [_vp, _vp, _vp, _vp, _i64, _vp],
    "pp_mlp_set_state": [_vp, _vp, _vp, _vp, _i64, _i64],
    "pp_mlp_features": [_vp, _vp, _vp, _vp, _i64, _vp, _vp],
    "pp_mlp_forward": [_vp, _vp, _vp, _i64, _vp, _vp],
    "pp_mlp_gradients": [_vp, _vp, _vp, _vp, _i64, _vp, _vp],
    "pp_mlp_train_step": [_vp, _vp, _vp, _vp, _i64, C.c_float, _vp],
    "pp_mlp_train_step_rows": [_vp, _vp, _vp, _vp, _i64, _vp, _i64, C.c_float, _vp],
    "pp_mlp_loss": [_vp, _vp],
    "pp_mlp_dom_sums": [_vp, _vp, _i64, _vp, C.c_float, _vp, _vp, _vp],
    "pp_mlp_sync": [_vp],
    "pp_mlp_set_exact_silu": [_vp, _i32],
    "pp_mlp_set_activation": [_vp, _i32],
    "pp_mlp_near_pairs": [_vp, _vp, _i64, C.c_float, _i64, _vp, _vp, _vp],
    "pp_debug_philox": [_vp, _vp, _vp, _vp, _i64],
    "pp_debug_trace": [_vp, _u64, _vp, _i64, _vp, _i64, _i32, _vp, _vp, _vp, _vp],
    "pp_debug_first_hit": [_vp, _vp, _i64, _i32, _vp, _vp],
    "pp_debug_gemm": [_vp, _vp, _vp, _i32, _i32, _i32, _vp],
    "pp_debug_scatter": [_vp, _vp, _vp, _vp, _i64],
    "pp_measure_issue_rate": [_i32, _i32, _vp, _vp],
    "pp_set_hit_acceptance": [_vp, _vp, _i32],
    "pp_debug_wait_timeout": [_i32, _u64, _vp, _vp],
}
EXPORTS = tuple(_SIGS) + ("pp_last_error", "pp_strerror", "pp_server_last_error",
                          "pp_mlp_last_error")

for _name, _args in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = C.c_int
_lib.pp_last_error.argtypes = [_vp]
_lib.pp_last_error.restype = C.c_char_p
_lib.pp_strerror.argtypes = [C.c_int]
_lib.pp_strerror.restype = C.c_char_p
_lib.pp_server_last_error.argtypes = [_vp]
_lib.pp_server_last_error.restype = C.c_char_p
_lib.pp_mlp_last_error.argtypes = [_vp]
_lib.pp_mlp_last_error.restype = C.c_char_p


class PPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def _ptr(x):
    """Host numpy array -> pointer; torch tensor -> its data pointer;
    int -> itself; None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


# ---- the C entry points, same names --------------------------------------

def pp_strerror(code: int) -> str:
    return _lib.pp_strerror(code).decode()


def pp_last_error(ctx) -> str:
    return _lib.pp_last_error(ctx).decode()


def _call(name, ctx, *args):
    rc = getattr(_lib, name)(ctx, *args)
    if rc != PP_OK:
        msg = pp_last_error(ctx) if ctx else pp_strerror(rc)
        raise PPError(rc, f"{name}: {msg}")
    return rc


def pp_config_default() -> pp_config:
    cfg = pp_config()
    rc = _lib.pp_config_default(C.byref(cfg))
    if rc:
        raise PPError(rc, "pp_config_default")
    return cfg


def pp_create(cfg: pp_config):
    h = C.c_void_p()
    rc = _lib.pp_create(C.byref(cfg), C.byref(h))
    if rc:
        raise PPError(rc, f"pp_create: {pp_strerror(rc)}")
    return h.value


def pp_destroy(ctx):
    return _lib.pp_destroy(ctx)


def pp_load_geometry(ctx, xyz, string_id, n_dom, dom_radius):
    return _call("pp_load_geometry", ctx, _ptr(xyz), _ptr(string_id), n_dom, dom_radius)


def pp_load_ice(ctx, b_e, a, n_layers, depth_top_m, dz_m, g):
    return _call("pp_load_ice", ctx, _ptr(b_e), _ptr(a), n_layers, depth_top_m, dz_m, g)


def pp_propagate(ctx, event_id, src, n_src, hits, counts):
    return _call("pp_propagate", ctx, event_id, _ptr(src), n_src, _ptr(hits), _ptr(counts))


def pp_propagate_batch(ctx, n_events, event_ids, src_begin, src, hits, counts):
    return _call("pp_propagate_batch", ctx, n_events, _ptr(event_ids), _ptr(src_begin),
                 _ptr(src), _ptr(hits), _ptr(counts))


def pp_propagate_batch_async(ctx, n_events, d_event_ids, d_src_begin, d_src, n_src, d_hits,
                             d_counts, stream=None):
    return _call("pp_propagate_batch_async", ctx, n_events, _ptr(d_event_ids),
                 _ptr(d_src_begin), _ptr(d_src), n_src, _ptr(d_hits), _ptr(d_counts),
                 _ptr(stream))


def pp_propagate_plain_async(ctx, n_events, h_event_ids, h_src_begin, h_event_photons, d_src,
                             d_hits, d_counts, stream=None):
    return _call("pp_propagate_plain_async", ctx, n_events, _ptr(h_event_ids),
                 _ptr(h_src_begin), _ptr(h_event_photons), _ptr(d_src), _ptr(d_hits),
                 _ptr(d_counts), _ptr(stream))


def pp_propagate_range_async(ctx, event_id, d_src, n_src, photon_begin, photon_end, accumulate,
                             d_hits, d_counts, stream=None):
    return _call("pp_propagate_range_async", ctx, event_id, _ptr(d_src), n_src, photon_begin,
                 photon_end, 1 if accumulate else 0, _ptr(d_hits), _ptr(d_counts), _ptr(stream))


# pp_hit: DOM index, source index, time (ns), weight
HIT_DTYPE = np.dtype([("dom", "<u4"), ("source", "<u4"), ("time_ns", "<f4"), ("weight", "<f4")])


def pp_propagate_records_async(ctx, n_events, d_event_ids, d_src_begin, d_src, n_src, d_hits,
                               d_counts, group_index, d_records, max_records, d_n_records,
                               stream=None):
    """Batched propagation that also writes compact hit records (16 bytes each,
    HIT_DTYPE) into d_records and their total number into d_n_records."""
    return _call("pp_propagate_records_async", ctx, n_events, _ptr(d_event_ids),
                 _ptr(d_src_begin), _ptr(d_src), n_src, _ptr(d_hits), _ptr(d_counts),
                 group_index, _ptr(d_records), max_records, _ptr(d_n_records), _ptr(stream))


PP_NOALLOC_MAX_SOURCES = 8192


def pp_propagate_noalloc(ctx, event_id, d_src, n_src, d_hits, d_counts, stream=None):
    """One event on device data; the library allocates nothing during the call
    (its scratch is a fixed static device array, at most 8192 sources)."""
    return _call("pp_propagate_noalloc", ctx, event_id, _ptr(d_src), n_src, _ptr(d_hits),
                 _ptr(d_counts), _ptr(stream))


def pp_sync(ctx, stream=None):
    return _call("pp_sync", ctx, _ptr(stream))


def pp_set_launch(ctx, block_threads=0, blocks_per_sm=0, refill_threshold=0, photons_per_lane=0):
    return _call("pp_set_launch", ctx, block_threads, blocks_per_sm, refill_threshold,
                 photons_per_lane)


def pp_autotune_batch(ctx, n_events, d_event_ids, d_src_begin, d_src, n_src, d_hits, d_counts,
                      stream=None, repeats=2):
    """-> ((block_threads, blocks_per_sm, refill_threshold, photons_per_lane), best_ms)"""
    best = (C.c_int32 * 4)()
    ms = C.c_float()
    _call("pp_autotune_batch", ctx, n_events, _ptr(d_event_ids), _ptr(d_src_begin), _ptr(d_src),
          n_src, _ptr(d_hits), _ptr(d_counts), _ptr(stream), repeats, C.addressof(best),
          C.addressof(ms))
    return tuple(best), ms.value


def pp_get_launch(ctx):
    """-> (block_threads, blocks_per_sm, refill_threshold, photons_per_lane, grid_blocks)"""
    v = [C.c_int32() for _ in range(5)]
    _call("pp_get_launch", ctx, *[C.addressof(x) for x in v])
    return tuple(x.value for x in v)


def pp_get_world(ctx):
    out = np.zeros(3, np.float32)
    _call("pp_get_world", ctx, _ptr(out))
    return tuple(float(v) for v in out)


def pp_set_graphs(ctx, enable):
    return _call("pp_set_graphs", ctx, 1 if enable else 0)


def pp_set_kernel_timing(ctx, enable):
    return _call("pp_set_kernel_timing", ctx, 1 if enable else 0)


def pp_get_kernel_time(ctx):
    """-> (total_ms, n_timed_launches, n_kernels_launched) since the last call."""
    ms, nt, nk = C.c_double(), C.c_uint64(), C.c_uint64()
    _call("pp_get_kernel_time", ctx, C.addressof(ms), C.addressof(nt), C.addressof(nk))
    return ms.value, nt.value, nk.value


def pp_get_memory(ctx):
    """(device bytes held by the context's buffers, device allocations made)."""
    b, n = C.c_uint64(0), C.c_uint64(0)
    _call("pp_get_memory", ctx, C.addressof(b), C.addressof(n))
    return b.value, n.value


def pp_get_path_stats(ctx):
    """-> (steps, layer crossings, photons born, steps with a string search)
    counted by the persistent kernel since the last call."""
    out = np.zeros(4, np.uint64)
    _call("pp_get_path_stats", ctx, _ptr(out))
    return int(out[0]), int(out[1]), int(out[2]), int(out[3])


def pp_debug_philox(ctx, ctr, key, out, n):
    return _call("pp_debug_philox", ctx, _ptr(ctr), _ptr(key), _ptr(out), n)


def pp_debug_trace(ctx, event_id, src, n_src, photon_ids, n, n_trace, outcome, n_steps, birth,
                   trace):
    return _call("pp_debug_trace", ctx, event_id, _ptr(src), n_src, _ptr(photon_ids), n,
                 n_trace, _ptr(outcome), _ptr(n_steps), _ptr(birth), _ptr(trace))


def pp_debug_scatter(ctx, dir, words, out, n):
    return _call("pp_debug_scatter", ctx, _ptr(dir), _ptr(words), _ptr(out), n)


def pp_debug_gemm(ctx, A, B, M, N, K, C):
    return _call("pp_debug_gemm", ctx, _ptr(A), _ptr(B), M, N, K, _ptr(C))


PP_MAX_ACCEPT_COEFFS = 8


def pp_set_hit_acceptance(ctx, coeffs):
    """Hit-record weights: clamp(sum c_i eta^i, 0, 1), eta = the direction's z at
    the DOM; an empty list restores weight 1."""
    c = np.ascontiguousarray(coeffs if coeffs is not None else [], np.float32)
    return _call("pp_set_hit_acceptance", ctx, _ptr(c) if c.size else None, int(c.size))


def pp_debug_wait_timeout(device, limit_ns):
    """(timed_out, waited_ns) of a bounded mbarrier wait that nothing completes."""
    flag, ns = C.c_int32(), C.c_uint64()
    rc = _lib.pp_debug_wait_timeout(device, limit_ns, C.byref(flag), C.byref(ns))
    if rc:
        raise PPError(rc, f"pp_debug_wait_timeout: {pp_strerror(rc)}")
    return flag.value, ns.value


PP_ISSUE_FP32_FMA, PP_ISSUE_SFU_LG2 = 0, 1


def pp_measure_issue_rate(device, kind):
    """(lane operations per second, timed launch in ms) of one pipe."""
    rate, ms = C.c_double(), C.c_double()
    rc = _lib.pp_measure_issue_rate(device, kind, C.byref(rate), C.byref(ms))
    if rc:
        raise PPError(rc, f"pp_measure_issue_rate: {pp_strerror(rc)}")
    return rate.value, ms.value


def bf16_bits(x) -> np.ndarray:
    """float array -> BF16 bit patterns (round to nearest even), uint16."""
    f = np.ascontiguousarray(x, np.float32).view(np.uint32)
    r = ((f >> 16) & 1) + 0x7FFF
    return ((f + r) >> 16).astype(np.uint16)


def bf16_value(bits) -> np.ndarray:
    """BF16 bit patterns -> float32 values."""
    return (np.asarray(bits, np.uint16).astype(np.uint32) << 16).view(np.float32)


def pp_debug_first_hit(ctx, seg, n, mode, dom, t):
    return _call("pp_debug_first_hit", ctx, _ptr(seg), n, mode, _ptr(dom), _ptr(t))


# ---- serving loop ------------------------------------------------------------

class pp_server_config(C.Structure):
    _fields_ = [("budget_bytes", C.c_uint64), ("arena_sources", C.c_int64),
                ("ring_requests", C.c_int32), ("idle_exit_us", C.c_int32),
                ("max_launch_ms", C.c_int32)]


def pp_server_config_default() -> pp_server_config:
    cfg = pp_server_config()
    rc = _lib.pp_server_config_default(C.byref(cfg))
    if rc:
        raise PPError(rc, "pp_server_config_default")
    return cfg


def pp_server_create(ctx, cfg: pp_server_config):
    h = C.c_void_p()
    rc = _lib.pp_server_create(ctx, C.byref(cfg), C.byref(h))
    if rc:
        raise PPError(rc, f"pp_server_create: {pp_last_error(ctx)}")
    return h.value


def pp_server_destroy(server):
    return _lib.pp_server_destroy(server)


def pp_server_last_error(server) -> str:
    return _lib.pp_server_last_error(server).decode()


def pp_submit(server, event_id, src, n_src):
    """-> ticket"""
    t = C.c_uint64()
    rc = _lib.pp_submit(server, event_id, _ptr(src), n_src, C.byref(t))
    if rc:
        raise PPError(rc, f"pp_submit: {pp_strerror(rc)}: {pp_server_last_error(server)}")
    return t.value


def pp_collect(server, ticket, hits, counts, timeout_ms=-1):
    """Returns the status code (PP_OK, PP_ETIMEDOUT, ...) without raising."""
    return _lib.pp_collect(server, ticket, _ptr(hits), _ptr(counts), timeout_ms)


def pp_server_stats(server):
    out = np.zeros(8)
    rc = _lib.pp_server_stats(server, _ptr(out))
    if rc:
        raise PPError(rc, "pp_server_stats")
    keys = ("bunches", "photons", "p50_ms", "p99_ms", "photons_per_s", "kernel_launches",
            "peak_admitted_bytes", "device_bytes")
    return dict(zip(keys, out.tolist()))


class Server:
    """A serving loop on a Propagator's context (same calls, numpy inputs)."""

    def __init__(self, prop, budget_bytes=None, arena_sources=None, ring_requests=None,
                 idle_exit_us=None, max_launch_ms=None):
        cfg = pp_server_config_default()
        for k, v in (("budget_bytes", budget_bytes), ("arena_sources", arena_sources),
                     ("ring_requests", ring_requests), ("idle_exit_us", idle_exit_us),
                     ("max_launch_ms", max_launch_ms)):
            if v is not None:
                setattr(cfg, k, v)
        self.prop = prop
        self.n_dom = prop.n_dom
        self.handle = pp_server_create(prop.ctx, cfg)

    def submit(self, event_id, sources):
        s = np.ascontiguousarray(sources)
        return pp_submit(self.handle, int(event_id), s if s.size else None, s.shape[0])

    def collect(self, ticket, timeout_ms=-1):
        """-> (status, hits [n_dom], counts [4])"""
        hits = np.zeros(self.n_dom, np.uint64)
        counts = np.zeros(4, np.uint64)
        rc = pp_collect(self.handle, ticket, hits, counts, timeout_ms)
        return rc, hits, counts

    def stats(self):
        return pp_server_stats(self.handle)

    def close(self):
        if self.handle:
            pp_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- learned surrogate ---------------------------------------------------------

PP_MLP_N_PARAMS = 206081
PP_MLP_INPUTS = 32


def _mcall(name, m, *args):
    rc = getattr(_lib, name)(m, *args)
    if rc != PP_OK:
        raise PPError(rc, f"{name}: {_lib.pp_mlp_last_error(m).decode() if m else pp_strerror(rc)}")
    return rc


def pp_mlp_create(ctx, max_batch, max_rows):
    h = C.c_void_p()
    rc = _lib.pp_mlp_create(ctx, max_batch, max_rows, C.byref(h))
    if rc:
        raise PPError(rc, f"pp_mlp_create: {pp_last_error(ctx)}")
    return h.value


def pp_mlp_last_error(m) -> str:
    return _lib.pp_mlp_last_error(m).decode()


def pp_mlp_destroy(m):
    return _lib.pp_mlp_destroy(m)


def pp_mlp_set_params(m, params, n):
    return _mcall("pp_mlp_set_params", m, _ptr(params), n)


def pp_mlp_get_params(m, params, n):
    return _mcall("pp_mlp_get_params", m, _ptr(params), n)


def pp_mlp_get_state(m, params, m1, v1, n):
    """Returns the Adam step count; fills params (and m1, v1 unless None)."""
    step = C.c_int64(0)
    _mcall("pp_mlp_get_state", m, _ptr(params), _ptr(m1), _ptr(v1), n, C.addressof(step))
    return step.value


def pp_mlp_set_state(m, params, m1, v1, n, step):
    return _mcall("pp_mlp_set_state", m, _ptr(params), _ptr(m1), _ptr(v1), n, step)


def pp_mlp_features(m, d_src, d_pair_src, d_pair_dom, n, d_feat, stream=None):
    return _mcall("pp_mlp_features", m, _ptr(d_src), _ptr(d_pair_src), _ptr(d_pair_dom), n,
                  _ptr(d_feat), _ptr(stream))


def pp_mlp_forward(m, d_feat, d_nph, n, d_lambda, stream=None):
    return _mcall("pp_mlp_forward", m, _ptr(d_feat), _ptr(d_nph), n, _ptr(d_lambda), _ptr(stream))


def pp_mlp_gradients(m, d_feat, d_nph, d_count, n, h_grads, h_loss):
    return _mcall("pp_mlp_gradients", m, _ptr(d_feat), _ptr(d_nph), _ptr(d_count), n,
                  _ptr(h_grads), _ptr(h_loss))


def pp_mlp_train_step(m, d_feat, d_nph, d_count, n, lr, stream=None):
    return _mcall("pp_mlp_train_step", m, _ptr(d_feat), _ptr(d_nph), _ptr(d_count), n, lr,
                  _ptr(stream))


def pp_mlp_train_step_rows(m, d_feat, d_nph, d_count, n_rows, d_rows, n, lr, stream=None):
    return _mcall("pp_mlp_train_step_rows", m, _ptr(d_feat), _ptr(d_nph), _ptr(d_count), n_rows,
                  _ptr(d_rows), n, lr, _ptr(stream))


def pp_mlp_loss(m):
    v = C.c_double()
    _mcall("pp_mlp_loss", m, C.addressof(v))
    return v.value


def pp_mlp_dom_sums(m, d_src, n_src, d_nph_src, r_max, d_dom_sums, d_lambda=None, stream=None):
    return _mcall("pp_mlp_dom_sums", m, _ptr(d_src), n_src, _ptr(d_nph_src), r_max,
                  _ptr(d_dom_sums), _ptr(d_lambda), _ptr(stream))


def pp_mlp_near_pairs(m, d_src, n_src, r_max, max_out, d_pair_src, d_pair_dom):
    """-> number of pairs within r_max (the first max_out are written)"""
    c = C.c_uint64()
    _mcall("pp_mlp_near_pairs", m, _ptr(d_src), n_src, r_max, max_out, _ptr(d_pair_src),
           _ptr(d_pair_dom), C.addressof(c))
    return c.value


def pp_mlp_sync(m):
    return _mcall("pp_mlp_sync", m)


PP_MLP_ACT_SILU, PP_MLP_ACT_HARD_SWISH = 0, 1


def pp_mlp_set_activation(m, act):
    return _mcall("pp_mlp_set_activation", m, act)


def pp_mlp_set_exact_silu(m, exact):
    return _mcall("pp_mlp_set_exact_silu", m, 1 if exact else 0)


def mlp_init_params(seed: int = 0) -> np.ndarray:
    """Initial parameters: weights N(0, 1/fan_in) (He-like for SiLU), zero
    biases, b5 chosen so that softplus(b5) is a small hit probability."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, np.sqrt(1.0 / PP_MLP_INPUTS), (256, PP_MLP_INPUTS)), np.zeros(256)]
    for _ in range(3):
        parts += [rng.normal(0.0, np.sqrt(2.0 / 256), (256, 256)), np.zeros(256)]
    parts += [rng.normal(0.0, np.sqrt(1.0 / 256), 256), np.array([-9.0])]
    p = np.concatenate([x.ravel() for x in parts]).astype(np.float32)
    assert p.size == PP_MLP_N_PARAMS
    return p


class Mlp:
    """The surrogate on a Propagator's context (device buffers are torch tensors)."""

    def __init__(self, prop, max_batch=16384, max_rows=1 << 18):
        self.prop = prop
        self.n_dom = prop.n_dom
        self.handle = pp_mlp_create(prop.ctx, max_batch, max_rows)

    def close(self):
        if self.handle:
            pp_mlp_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_activation(self, act):
        """PP_MLP_ACT_SILU or PP_MLP_ACT_HARD_SWISH (or "silu" / "hswish")."""
        codes = {"silu": PP_MLP_ACT_SILU, "hswish": PP_MLP_ACT_HARD_SWISH}
        pp_mlp_set_activation(self.handle, codes.get(act, act))

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        pp_mlp_set_params(self.handle, p, p.size)

    def get_params(self):
        p = np.zeros(PP_MLP_N_PARAMS, np.float32)
        pp_mlp_get_params(self.handle, p, p.size)
        return p


# ---- convenience wrapper ---------------------------------------------------

class Propagator:
    """One library context with geometry and ice loaded."""

    def __init__(self, geom, ice, seed=0, device=0, max_steps=100_000, world_margin=100.0,
                 depth_of_z0=1950.0, scatter_coeff_is_effective=True, stream=None):
        cfg = pp_config_default()
        cfg.device = device
        cfg.seed = seed
        cfg.max_steps = max_steps
        cfg.world_margin_m = world_margin
        cfg.depth_of_z0_m = depth_of_z0
        cfg.scatter_coeff_is_effective = 1 if scatter_coeff_is_effective else 0
        cfg.stream = _ptr(stream)
        self.stream = cfg.stream    # the context's stream handle (None: its own)
        self.ctx = pp_create(cfg)
        self.n_dom = geom.n_dom
        xyz = np.ascontiguousarray(geom.xyz, np.float32).reshape(-1, 3)
        self.geom_xyz = xyz.astype(np.float64)
        sid = np.ascontiguousarray(geom.string_id, np.int32)
        pp_load_geometry(self.ctx, xyz if xyz.size else None, sid if sid.size else None,
                         geom.n_dom, float(geom.dom_radius))
        b_e = np.ascontiguousarray(ice.b_e, np.float32)
        a = np.ascontiguousarray(ice.a, np.float32)
        pp_load_ice(self.ctx, b_e, a, ice.n_layers, float(ice.depth_top), float(ice.dz),
                    float(ice.g))

    def close(self):
        if self.ctx:
            pp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @staticmethod
    def _src(sources):
        s = np.ascontiguousarray(sources)
        if s.dtype != workloads.SOURCE_DTYPE:
            raise TypeError("sources must use workloads.SOURCE_DTYPE")
        return s

    def propagate(self, event_id, sources):
        """Plain path for one event: (hits [n_dom], counts [4])."""
        s = self._src(sources)
        hits = np.zeros(self.n_dom, np.uint64)
        counts = np.zeros(4, np.uint64)
        pp_propagate(self.ctx, int(event_id), s if s.size else None, s.shape[0], hits, counts)
        return hits, counts

    def propagate_batch(self, batch):
        """Persistent batched path: (hits [E, n_dom], counts [E, 4])."""
        s = self._src(batch.sources)
        ids = np.ascontiguousarray(batch.event_ids, np.uint64)
        beg = np.ascontiguousarray(batch.src_begin, np.int64)
        E = ids.shape[0]
        hits = np.zeros((E, self.n_dom), np.uint64)
        counts = np.zeros((E, 4), np.uint64)
        pp_propagate_batch(self.ctx, E, ids, beg, s if s.size else None, hits, counts)
        return hits, counts

    def set_launch(self, block_threads=0, blocks_per_sm=0, refill_threshold=0, photons_per_lane=0):
        pp_set_launch(self.ctx, block_threads, blocks_per_sm, refill_threshold, photons_per_lane)

    def get_launch(self):
        return pp_get_launch(self.ctx)

    def world(self):
        return pp_get_world(self.ctx)

    def philox(self, ctr, key):
        ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
        key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, np.uint32).reshape(-1, 2),
                                                   (ctr.shape[0], 2)))
        out = np.zeros_like(ctr)
        pp_debug_philox(self.ctx, ctr, key, out, ctr.shape[0])
        return out

    def trace(self, event_id, sources, photon_ids, n_trace=10):
        s = self._src(sources)
        ids = np.ascontiguousarray(photon_ids, np.uint64).ravel()
        n = ids.shape[0]
        outc = np.zeros(n, np.int32)
        ns = np.zeros(n, np.int64)
        birth = np.zeros((n, 6), np.float32)
        tr = np.zeros((n, max(n_trace, 0), 3), np.float32)
        pp_debug_trace(self.ctx, int(event_id), s, s.shape[0], ids, n, n_trace, outc, ns, birth,
                       tr if n_trace > 0 else None)
        return outc, ns, birth, tr

    def scatter(self, d, words):
        d = np.ascontiguousarray(d, np.float32).reshape(-1, 3)
        words = np.ascontiguousarray(words, np.uint32).reshape(-1, 2)
        out = np.zeros_like(d)
        pp_debug_scatter(self.ctx, d, words, out, d.shape[0])
        return out

    def first_hit(self, p, d, S, mode=0):
        p = np.asarray(p, np.float32).reshape(-1, 3)
        S = np.broadcast_to(np.asarray(S, np.float32), (p.shape[0],)).reshape(-1, 1)
        seg = np.ascontiguousarray(np.concatenate(
            [p, np.asarray(d, np.float32).reshape(-1, 3), S], axis=1), np.float32)
        n = seg.shape[0]
        dom = np.zeros(n, np.int32)
        t = np.zeros(n, np.float32)
        pp_debug_first_hit(self.ctx, seg, n, mode, dom, t)
        return dom, t
