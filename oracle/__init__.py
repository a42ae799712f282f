"""CPU oracle for the photon-propagation path (ctypes binding of oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library's product path.
It shares no code with the CUDA library and does not import it.

Every function here marshals numpy arrays into the plain C entry points of
``oracle.cpp``; the arithmetic lives there, in double precision.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

OUT_ABSORBED, OUT_ESCAPED, OUT_TRUNCATED = -1, -2, -3


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (g++, C++17, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [
        ("seed", C.c_uint64), ("max_steps", C.c_uint32),
        ("scatter_coeff_is_effective", C.c_int32),
        ("g", C.c_double), ("world_margin", C.c_double), ("depth_of_z0", C.c_double),
        ("n_dom", C.c_int32), ("brute_force", C.c_int32), ("dom_radius", C.c_double),
        ("dom_xyz", C.c_void_p), ("string_id", C.c_void_p),
        ("n_layers", C.c_int32), ("n_threads", C.c_int32),
        ("depth_top", C.c_double), ("layer_dz", C.c_double),
        ("b_e", C.c_void_p), ("a", C.c_void_p),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        P = C.POINTER(Params)
        vp, i64, i32, d = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        sig = {
            "orc_philox": ([vp, vp, vp, i64], None),
            "orc_u01": ([vp, vp, i64], None),
            "orc_hg": ([d, vp, vp, i64], None),
            "orc_rotate": ([vp, vp, vp, vp, i64], None),
            "orc_layer_at": ([P, vp, vp, vp, i64], None),
            "orc_walk": ([P, vp, vp, vp, vp, vp, vp, vp, vp, i64], None),
            "orc_world_exit": ([P, vp, vp, vp, i64], None),
            "orc_world": ([P, vp], None),
            "orc_first_hit": ([P, vp, vp, vp, vp, vp, i64], None),
            "orc_propagate": ([P, i32, vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
            "orc_trace": ([P, C.c_uint64, i64, vp, vp, vp, vp, i64, i32, vp, vp, vp, vp, vp], C.c_int),
            "orc_hit_records": ([P, C.c_uint64, i64, vp, vp, vp, d, C.c_int32, vp, i64, vp, vp,
                                 vp, vp, vp, vp], C.c_int),
        }
        for name, (args, res) in sig.items():
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = res
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Model:
    """Geometry + ice + run settings, in the form oracle.cpp takes.  Keeps the
    numpy arrays alive for as long as the ctypes struct points at them."""

    def __init__(self, geom, ice, seed=0, max_steps=100_000, world_margin=100.0,
                 depth_of_z0=1950.0, scatter_coeff_is_effective=True, brute_force=False,
                 n_threads=0):
        self.xyz = np.ascontiguousarray(geom.xyz, dtype=np.float32).reshape(-1, 3)
        self.sid = np.ascontiguousarray(geom.string_id, dtype=np.int32)
        self.b_e = np.ascontiguousarray(ice.b_e, dtype=np.float32)
        self.a = np.ascontiguousarray(ice.a, dtype=np.float32)
        p = Params()
        p.seed = seed
        p.max_steps = max_steps
        p.scatter_coeff_is_effective = 1 if scatter_coeff_is_effective else 0
        p.g = float(ice.g)
        p.world_margin = float(world_margin)
        p.depth_of_z0 = float(depth_of_z0)
        p.n_dom = self.xyz.shape[0]
        p.brute_force = 1 if brute_force else 0
        p.dom_radius = float(geom.dom_radius)
        p.dom_xyz = _ptr(self.xyz).value if self.xyz.size else None
        p.string_id = _ptr(self.sid).value if self.sid.size else None
        p.n_layers = self.b_e.shape[0]
        p.n_threads = n_threads
        p.depth_top = float(ice.depth_top)
        p.layer_dz = float(ice.dz)
        p.b_e = _ptr(self.b_e).value
        p.a = _ptr(self.a).value
        self.p = p

    def pref(self):
        return C.byref(self.p)


# ----------------------------------------------------------------- primitives

def philox(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    key = np.ascontiguousarray(np.broadcast_to(np.asarray(key, np.uint32).reshape(-1, 2),
                                               (ctr.shape[0], 2)))
    out = np.zeros_like(ctr)
    lib().orc_philox(_ptr(ctr), _ptr(key), _ptr(out), ctr.shape[0])
    return out


def u01(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.uint32).ravel()
    u = np.zeros(x.shape[0], np.float64)
    lib().orc_u01(_ptr(x), _ptr(u), x.shape[0])
    return u


def hg(g: float, u: np.ndarray) -> np.ndarray:
    u = np.ascontiguousarray(u, dtype=np.float64).ravel()
    mu = np.zeros_like(u)
    lib().orc_hg(float(g), _ptr(u), _ptr(mu), u.shape[0])
    return mu


def rotate(d, mu, phi) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    mu = np.ascontiguousarray(mu, dtype=np.float64).ravel()
    phi = np.ascontiguousarray(phi, dtype=np.float64).ravel()
    out = np.zeros_like(d)
    lib().orc_rotate(_ptr(d), _ptr(mu), _ptr(phi), _ptr(out), d.shape[0])
    return out


def layer_at(model: Model, z, w) -> np.ndarray:
    z = np.ascontiguousarray(z, dtype=np.float64).ravel()
    w = np.ascontiguousarray(np.broadcast_to(w, z.shape), dtype=np.float64)
    out = np.zeros(z.shape[0], np.int32)
    lib().orc_layer_at(model.pref(), _ptr(z), _ptr(w), _ptr(out), z.shape[0])
    return out


def walk(model: Model, z, w, tau_s, tau_a):
    z = np.ascontiguousarray(z, dtype=np.float64).ravel()
    n = z.shape[0]
    w = np.ascontiguousarray(np.broadcast_to(w, (n,)), dtype=np.float64)
    ts = np.ascontiguousarray(np.broadcast_to(tau_s, (n,)), dtype=np.float64)
    ta = np.ascontiguousarray(np.broadcast_to(tau_a, (n,)), dtype=np.float64)
    S = np.zeros(n)
    ab = np.zeros(n, np.int32)
    le = np.zeros(n, np.int32)
    tae = np.zeros(n)
    lib().orc_walk(model.pref(), _ptr(z), _ptr(w), _ptr(ts), _ptr(ta), _ptr(S), _ptr(ab),
                   _ptr(le), _ptr(tae), n)
    return S, ab.astype(bool), le, tae


def world(model: Model):
    out = np.zeros(3)
    lib().orc_world(model.pref(), _ptr(out))
    return tuple(out)


def world_exit(model: Model, p, d) -> np.ndarray:
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    t = np.zeros(p.shape[0])
    lib().orc_world_exit(model.pref(), _ptr(p), _ptr(d), _ptr(t), p.shape[0])
    return t


def first_hit(model: Model, p, d, S):
    p = np.ascontiguousarray(p, dtype=np.float64).reshape(-1, 3)
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    S = np.ascontiguousarray(np.broadcast_to(S, (p.shape[0],)), dtype=np.float64)
    dom = np.zeros(p.shape[0], np.int32)
    t = np.zeros(p.shape[0])
    lib().orc_first_hit(model.pref(), _ptr(p), _ptr(d), _ptr(S), _ptr(dom), _ptr(t), p.shape[0])
    return dom, t


# ------------------------------------------------------------- propagation --

def _source_arrays(sources):
    f = np.stack([sources[k].astype(np.float32) for k in
                  ("x", "y", "z", "dx", "dy", "dz", "length")], axis=1)
    f = np.ascontiguousarray(f, dtype=np.float32)
    typ = np.ascontiguousarray(sources["type"], dtype=np.uint32)
    nph = np.ascontiguousarray(sources["n_photons"], dtype=np.uint64)
    return f, typ, nph


def propagate(model: Model, batch):
    """All photons of all events of ``batch``.  Returns (hits [E, n_dom] u64,
    counts [E, 4] u64 = absorbed, escaped, truncated, steps, stats dict)."""
    f, typ, nph = _source_arrays(batch.sources)
    ev = np.ascontiguousarray(batch.event_ids, dtype=np.uint64)
    beg = np.ascontiguousarray(batch.src_begin, dtype=np.int64)
    E = ev.shape[0]
    hits = np.zeros((E, model.p.n_dom), np.uint64)
    counts = np.zeros((E, 4), np.uint64)
    stats = np.zeros(4)
    rc = lib().orc_propagate(model.pref(), E, _ptr(ev), _ptr(beg), _ptr(f), _ptr(typ),
                             _ptr(nph), _ptr(hits), _ptr(counts), _ptr(stats))
    if rc != 0:
        raise RuntimeError(f"orc_propagate failed: {rc}")
    return hits, counts, {"scatters": stats[0], "crossings": stats[1], "path": stats[2],
                          "cos_sum": stats[3]}


def trace(model: Model, event_id: int, sources, photon_ids, n_trace: int = 10,
          margins: bool = False):
    """Follows chosen photons of one event.  Returns (outcome [n] i32,
    n_steps [n] i64, birth [n, 6], trace [n, n_trace, 3]) and, with
    margins=True, also the per-step decision margins [n, n_trace] (metres)."""
    f, typ, nph = _source_arrays(sources)
    ids = np.ascontiguousarray(photon_ids, dtype=np.uint64).ravel()
    n = ids.shape[0]
    outc = np.zeros(n, np.int32)
    ns = np.zeros(n, np.int64)
    birth = np.zeros((n, 6))
    tr = np.zeros((n, n_trace, 3))
    mg = np.zeros((n, n_trace)) if margins else None
    rc = lib().orc_trace(model.pref(), int(event_id), f.shape[0], _ptr(f), _ptr(typ), _ptr(nph),
                         _ptr(ids), n, n_trace, _ptr(outc), _ptr(ns), _ptr(birth), _ptr(tr),
                         _ptr(mg) if margins else None)
    if rc != 0:
        raise RuntimeError(f"orc_trace failed: {rc}")
    if margins:
        return outc, ns, birth, tr, mg
    return outc, ns, birth, tr


def hit_records(model: Model, event_id: int, sources, group_index: float = 1.35,
                max_records: int = 1 << 22, acceptance=None):
    """Compact hit records of one event (single-threaded): dict of arrays
    dom (u32), source (u32), time_ns (f64), weight (f64), photon (u64,
    per-event id).  acceptance: polynomial coefficients c_0.. in the z
    component of the photon's direction at the DOM (weight = clamp to [0, 1]
    of sum c_i eta^i); None gives weight 1."""
    f, typ, nph = _source_arrays(sources)
    acc = np.ascontiguousarray([] if acceptance is None else acceptance, np.float64)
    dom = np.zeros(max_records, np.uint32)
    src = np.zeros(max_records, np.uint32)
    t = np.zeros(max_records)
    w = np.zeros(max_records)
    ph = np.zeros(max_records, np.uint64)
    n = C.c_int64()
    rc = lib().orc_hit_records(model.pref(), int(event_id), f.shape[0], _ptr(f), _ptr(typ),
                               _ptr(nph), float(group_index), int(acc.size),
                               _ptr(acc) if acc.size else None, max_records, _ptr(dom),
                               _ptr(src), _ptr(t), _ptr(w), _ptr(ph), C.addressof(n))
    if rc != 0:
        raise RuntimeError(f"orc_hit_records failed: {rc}")
    k = min(n.value, max_records)
    return {"dom": dom[:k], "source": src[:k], "time_ns": t[:k], "weight": w[:k],
            "photon": ph[:k], "n": n.value}
