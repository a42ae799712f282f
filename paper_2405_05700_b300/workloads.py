"""Seeded synthetic inputs for the photon-propagation path.

This module only *builds inputs*: detector geometry, ice-property tables and
photon sources.  It holds none of the propagation arithmetic, imports neither
the CUDA binding nor the oracle, and is the one module both sides are fed from.

Workloads follow the setting the paper gives for IceCube's photon propagation
step (Sec. 1 and Sec. 2): 5160 DOMs between 1450 m and 2450 m depth, ice in
10 m layers with per-layer scattering and absorption, light sources handed on
as photon-emitting steps (Sec. 4), primaries generated on a cylinder slightly
larger than the instrumented volume (Sec. 4).  The paper prints no workload
numbers for the propagator itself; the concrete recipes below are readings
of it, each stated in the docstring of the function that builds it
(coordinate convention, hex string layout, ice profiles, muon-bundle recipe).

Coordinates: right-handed, metres, z up, ``z = Z0_DEPTH - depth`` with
``Z0_DEPTH = 1950``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

Z0_DEPTH = 1950.0          # depth (m) of the z = 0 plane
STRING_SPACING = 125.0     # hex lattice pitch (m)
DOMS_PER_STRING = 60
DOM_SPACING = 17.0         # vertical pitch (m); DOM k sits at depth 1450 + 17 k
DOM_TOP_DEPTH = 1450.0
DOM_RADIUS = 0.1651        # m
LAYER_DZ = 10.0            # Sec. 2: ice described in 10 m layers
WORLD_MARGIN = 100.0       # world cylinder = DOM extent + this margin

SRC_ISO_POINT = 0
SRC_CHERENKOV = 1
SRC_CASCADE = 2

# One photon source ("photon emitting step", Sec. 4).  40 bytes, the same
# field order and widths as the library's C struct and the oracle's inputs.
SOURCE_DTYPE = np.dtype([
    ("x", "<f4"), ("y", "<f4"), ("z", "<f4"),
    ("dx", "<f4"), ("dy", "<f4"), ("dz", "<f4"),
    ("length", "<f4"), ("type", "<u4"), ("n_photons", "<u8"),
])
assert SOURCE_DTYPE.itemsize == 40


@dataclasses.dataclass
class Geometry:
    xyz: np.ndarray          # float32 [n_dom, 3]
    string_id: np.ndarray    # int32 [n_dom]
    dom_radius: float

    @property
    def n_dom(self) -> int:
        return int(self.xyz.shape[0])


@dataclasses.dataclass
class Ice:
    b_e: np.ndarray          # float32 [L] effective scattering coefficient (1/m)
    a: np.ndarray            # float32 [L] absorption coefficient (1/m)
    depth_top: float         # depth of the top of layer 0 (m)
    dz: float                # layer thickness (m)
    g: float                 # Henyey-Greenstein mean cosine

    @property
    def n_layers(self) -> int:
        return int(self.b_e.shape[0])


@dataclasses.dataclass
class Batch:
    """Many events' sources, concatenated; event e owns
    ``sources[src_begin[e]:src_begin[e+1]]``."""
    event_ids: np.ndarray    # uint64 [n_events]
    src_begin: np.ndarray    # int64 [n_events + 1]
    sources: np.ndarray      # SOURCE_DTYPE [n_src]

    @property
    def n_events(self) -> int:
        return int(self.event_ids.shape[0])

    def photons_per_event(self) -> np.ndarray:
        cs = np.concatenate([[0], np.cumsum(self.sources["n_photons"].astype(np.uint64))])
        return (cs[self.src_begin[1:]] - cs[self.src_begin[:-1]]).astype(np.uint64)

    def total_photons(self) -> int:
        return int(self.sources["n_photons"].astype(np.uint64).sum())

    def event(self, e: int) -> np.ndarray:
        return self.sources[self.src_begin[e]:self.src_begin[e + 1]]

    def select(self, events) -> "Batch":
        events = list(events)
        parts = [self.event(e) for e in events]
        begin = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).astype(np.int64)
        src = np.concatenate(parts) if parts else np.zeros(0, SOURCE_DTYPE)
        return Batch(self.event_ids[events].astype(np.uint64), begin, src)


# ---------------------------------------------------------------- geometry --

def hex_string_positions(n_strings: int) -> np.ndarray:
    """First ``n_strings`` points of an axial hex lattice (pitch 125 m) about
    the origin, ordered by (radius, polar angle in [0, 2 pi))."""
    pts = []
    rmax = 1
    while 3 * rmax * (rmax + 1) + 1 < n_strings:
        rmax += 1
    for q in range(-rmax, rmax + 1):
        for r in range(-rmax, rmax + 1):
            s = -q - r
            if max(abs(q), abs(r), abs(s)) > rmax:
                continue
            x = STRING_SPACING * (q + 0.5 * r)
            y = STRING_SPACING * (math.sqrt(3.0) / 2.0) * r
            rad = math.hypot(x, y)
            ang = math.atan2(y, x) % (2.0 * math.pi)
            pts.append((round(rad, 6), round(ang, 9), x, y))
    pts.sort()
    return np.array([(p[2], p[3]) for p in pts[:n_strings]], dtype=np.float64)


def make_geometry(n_strings: int, doms_per_string: int = DOMS_PER_STRING) -> Geometry:
    """Hex string grid; DOM k on a string at depth 1450 + 17 k (Sec. 1 puts the
    DOMs between 1450 m and 2450 m).  DOM index = string * 60 + k."""
    sxy = hex_string_positions(n_strings)
    k = np.arange(doms_per_string, dtype=np.float64)
    z = Z0_DEPTH - (DOM_TOP_DEPTH + DOM_SPACING * k)
    xyz = np.zeros((n_strings * doms_per_string, 3), dtype=np.float64)
    sid = np.zeros(n_strings * doms_per_string, dtype=np.int32)
    for s in range(n_strings):
        sl = slice(s * doms_per_string, (s + 1) * doms_per_string)
        xyz[sl, 0] = sxy[s, 0]
        xyz[sl, 1] = sxy[s, 1]
        xyz[sl, 2] = z
        sid[sl] = s
    return Geometry(xyz.astype(np.float32), sid, DOM_RADIUS)


def geometry_tiny() -> Geometry:
    """7 strings (centre + first ring) x 60 DOMs = 420 DOMs."""
    return make_geometry(7)


def geometry_full() -> Geometry:
    """86 strings x 60 DOMs = 5160 DOMs (the count Sec. 1 gives)."""
    return make_geometry(86)


def world_cylinder(geom: Geometry, margin: float = WORLD_MARGIN):
    """(radius, z_min, z_max) of the cylinder that bounds the simulated volume
    for workload construction (track clipping, generation surface)."""
    xyz = geom.xyz.astype(np.float64)
    if xyz.shape[0] == 0:
        return margin, -margin, margin
    r = float(np.max(np.hypot(xyz[:, 0], xyz[:, 1]))) + margin
    return r, float(xyz[:, 2].min()) - margin, float(xyz[:, 2].max()) + margin


# --------------------------------------------------------------------- ice --

def ice_tiny(seed: int = 0, n_layers: int = 100) -> Ice:
    """100 layers of 10 m from 1450 m: b_e ~ U[0.02, 0.1], a ~ U[0.005, 0.02]
    drawn i.i.d. (b_e array first, then a), HG g = 0.9."""
    rng = np.random.default_rng(seed)
    b_e = rng.uniform(0.02, 0.1, n_layers)
    a = rng.uniform(0.005, 0.02, n_layers)
    return Ice(b_e.astype(np.float32), a.astype(np.float32), 1450.0, LAYER_DZ, 0.9)


def ice_full(seed: int = 0, n_layers: int = 171, depth_top: float = 1100.0) -> Ice:
    """171 layers of 10 m from 1100 m: smooth seeded profiles evaluated at
    layer mid-depths, and the layer holding depth 2000 m scaled x3 (one dust
    layer)."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0.0, 2.0 * math.pi, 3)
    d = depth_top + LAYER_DZ * (np.arange(n_layers) + 0.5)
    b_e = 0.05 * (1.0 + 0.4 * np.sin(2 * np.pi * d / 300.0 + ph[0])
                  + 0.2 * np.sin(2 * np.pi * d / 97.0 + ph[1]))
    a = 0.0125 * (1.0 + 0.4 * np.sin(2 * np.pi * d / 250.0 + ph[2]))
    dust = int((2000.0 - depth_top) // LAYER_DZ)
    b_e[dust] *= 3.0
    a[dust] *= 3.0
    return Ice(b_e.astype(np.float32), a.astype(np.float32), depth_top, LAYER_DZ, 0.9)


def ice_homogeneous(b_e: float, a: float, g: float = 0.9, n_layers: int = 1,
                    depth_top: float = 0.0, dz: float = LAYER_DZ) -> Ice:
    return Ice(np.full(n_layers, b_e, np.float32), np.full(n_layers, a, np.float32),
               depth_top, dz, g)


# ----------------------------------------------------------------- sources --

def make_sources(n: int) -> np.ndarray:
    return np.zeros(n, dtype=SOURCE_DTYPE)


def point_source(x, y, z, n_photons, kind=SRC_ISO_POINT) -> np.ndarray:
    s = make_sources(1)
    s["x"], s["y"], s["z"] = x, y, z
    s["dz"] = 1.0
    s["type"] = kind
    s["n_photons"] = n_photons
    return s


def single_event(sources: np.ndarray, event_id: int = 0) -> Batch:
    return Batch(np.array([event_id], np.uint64),
                 np.array([0, len(sources)], np.int64), sources)


def sources_tiny(n_photons: int = 200_000) -> Batch:
    """One isotropic point source on the centre string at depth 1950 m."""
    return single_event(point_source(0.0, 0.0, 0.0, n_photons), 0)


def _clip_line_to_cylinder(p0, d, R, zlo, zhi):
    """Parameter interval [t0, t1] of the line p0 + t d inside the vertical
    cylinder, or None."""
    t0, t1 = -np.inf, np.inf
    a = d[0] ** 2 + d[1] ** 2
    if a > 0:
        b = p0[0] * d[0] + p0[1] * d[1]
        c = p0[0] ** 2 + p0[1] ** 2 - R * R
        disc = b * b - a * c
        if disc <= 0:
            return None
        sq = math.sqrt(disc)
        t0, t1 = (-b - sq) / a, (-b + sq) / a
    elif p0[0] ** 2 + p0[1] ** 2 > R * R:
        return None
    if d[2] != 0:
        za, zb = (zlo - p0[2]) / d[2], (zhi - p0[2]) / d[2]
        t0, t1 = max(t0, min(za, zb)), min(t1, max(za, zb))
    elif not (zlo <= p0[2] <= zhi):
        return None
    if t1 <= t0:
        return None
    return t0, t1


def _perp_basis(d):
    a = np.array([1.0, 0.0, 0.0]) if abs(d[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(d, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(d, e1)
    return e1, e2


def _muon_segments(p0, d, R, zlo, zhi, n_photons, seg_len=1.0):
    """Split the part of a straight muon track inside the world cylinder into
    1 m Cherenkov segments with ``n_photons`` spread evenly over them."""
    iv = _clip_line_to_cylinder(p0, d, R, zlo, zhi)
    if iv is None:
        return make_sources(0)
    t0, t1 = iv
    L = t1 - t0
    nseg = max(1, int(math.ceil(L / seg_len)))
    s = make_sources(nseg)
    ts = t0 + seg_len * np.arange(nseg)
    lens = np.minimum(seg_len, t1 - ts)
    s["x"] = p0[0] + ts * d[0]
    s["y"] = p0[1] + ts * d[1]
    s["z"] = p0[2] + ts * d[2]
    s["dx"], s["dy"], s["dz"] = d[0], d[1], d[2]
    s["length"] = lens
    s["type"] = SRC_CHERENKOV
    base, rem = divmod(int(n_photons), nseg)
    npk = np.full(nseg, base, np.uint64)
    npk[:rem] += 1
    s["n_photons"] = npk
    return s


def muon_bundle(rng, geom: Geometry, energy_gev: float, multiplicity: int,
                cos_zenith: float, azimuth: float, photons_per_gev: float = 10.0,
                lateral_sigma: float = 10.0, total_photons: int | None = None):
    """Sources of one downgoing muon bundle: axis drawn through the disc that
    covers the world cylinder (rejecting misses), muons offset laterally by a
    2-D Gaussian, each a straight line clipped to the world and cut into 1 m
    Cherenkov segments.  Photons: ``photons_per_gev * E`` (or
    ``total_photons``) split evenly over the muons."""
    R, zlo, zhi = world_cylinder(geom)
    zc = 0.5 * (zlo + zhi)
    st = math.sqrt(max(0.0, 1.0 - cos_zenith ** 2))
    d = -np.array([st * math.cos(azimuth), st * math.sin(azimuth), cos_zenith])
    e1, e2 = _perp_basis(d)
    rgen = math.hypot(R, 0.5 * (zhi - zlo))
    centre = np.array([0.0, 0.0, zc])
    for _ in range(1000):
        rr = rgen * math.sqrt(rng.uniform())
        ph = rng.uniform(0.0, 2.0 * math.pi)
        p_axis = centre + rr * (math.cos(ph) * e1 + math.sin(ph) * e2)
        if _clip_line_to_cylinder(p_axis, d, R, zlo, zhi) is not None:
            break
    ntot = int(round(photons_per_gev * energy_gev)) if total_photons is None else int(total_photons)
    base, rem = divmod(ntot, multiplicity)
    parts = []
    for m in range(multiplicity):
        off = rng.normal(0.0, lateral_sigma, 2)
        p = p_axis + off[0] * e1 + off[1] * e2
        parts.append(_muon_segments(p, d, R, zlo, zhi, base + (1 if m < rem else 0)))
    return np.concatenate(parts) if parts else make_sources(0)


def power_law_energy(rng, n, gamma=2.7, emin=1e3, emax=1e7):
    """Inverse-CDF draw from E^-gamma on [emin, emax]."""
    u = rng.uniform(size=n)
    k = 1.0 - gamma
    return (emin ** k + u * (emax ** k - emin ** k)) ** (1.0 / k)


def poisson_at_least_one(rng, mean, n):
    out = np.zeros(n, np.int64)
    for i in range(n):
        k = 0
        while k < 1:
            k = int(rng.poisson(mean))
        out[i] = k
    return out


def events_full(n_events: int = 1000, seed: int = 1, geom: Geometry | None = None,
                photons_per_gev: float = 10.0) -> Batch:
    """Power-law (E^-2.7, 1e3-1e7 GeV) downgoing muon bundles, cos zenith
    ~ U[0.3, 1], azimuth ~ U[0, 2 pi), multiplicity Poisson(3) >= 1,
    10 photons/GeV, 41 degree Cherenkov light from 1 m segments."""
    geom = geometry_full() if geom is None else geom
    rng = np.random.default_rng(seed)
    E = power_law_energy(rng, n_events)
    cz = rng.uniform(0.3, 1.0, n_events)
    az = rng.uniform(0.0, 2.0 * math.pi, n_events)
    mult = poisson_at_least_one(rng, 3.0, n_events)
    parts = []
    for e in range(n_events):
        parts.append(muon_bundle(rng, geom, E[e], int(mult[e]), cz[e], az[e], photons_per_gev))
    begin = np.concatenate([[0], np.cumsum([len(p) for p in parts])]).astype(np.int64)
    return Batch(np.arange(n_events, dtype=np.uint64), begin, np.concatenate(parts))


def event_large(total_photons: int = 10_000_000_000, seed: int = 5,
                geom: Geometry | None = None) -> Batch:
    """One 1e7 GeV bundle of 20 muons carrying ``total_photons`` photons."""
    geom = geometry_full() if geom is None else geom
    rng = np.random.default_rng(seed)
    src = muon_bundle(rng, geom, 1e7, 20, 0.8, 1.0, total_photons=total_photons)
    return single_event(src, 0)


def sources_gate(photons_per_dom: int = 1000, offset: float = 3.0,
                 geom: Geometry | None = None) -> Batch:
    """One isotropic point source ``offset`` metres from every DOM (along +x),
    so that nearly every DOM of the tiny detector is lit: the input of the
    per-DOM statistical comparison between two independent propagators."""
    geom = geometry_tiny() if geom is None else geom
    s = make_sources(geom.n_dom)
    s["x"] = geom.xyz[:, 0] + offset
    s["y"] = geom.xyz[:, 1]
    s["z"] = geom.xyz[:, 2]
    s["dz"] = 1.0
    s["type"] = SRC_ISO_POINT
    s["n_photons"] = photons_per_dom
    return single_event(s, 7)


def serving_bunch(rng, geom: Geometry | None = None, photons_min: float = 1e4,
                  photons_max: float = 1e7) -> np.ndarray:
    """Sources of one photon bunch of the serving workload: a downgoing muon
    track (cos zenith ~ U[0.3, 1]) through the world cylinder with stochastic
    energy losses -- cascades every U[5, 50] m with energies log-uniform in
    [1, 1e4] GeV.  The bunch carries a log-uniform number of photons in
    [photons_min, photons_max], split over the track's 1 m Cherenkov segments
    and its cascades (isotropic points) in proportion to segment length and
    cascade energy, 1 GeV of cascade energy weighing as 1 m of track."""
    geom = geometry_full() if geom is None else geom
    R, zlo, zhi = world_cylinder(geom)
    cz = rng.uniform(0.3, 1.0)
    az = rng.uniform(0.0, 2.0 * math.pi)
    st = math.sqrt(1.0 - cz * cz)
    d = -np.array([st * math.cos(az), st * math.sin(az), cz])
    e1, e2 = _perp_basis(d)
    rgen = math.hypot(R, 0.5 * (zhi - zlo))
    centre = np.array([0.0, 0.0, 0.5 * (zlo + zhi)])
    iv = None
    for _ in range(1000):
        rr = rgen * math.sqrt(rng.uniform())
        ph = rng.uniform(0.0, 2.0 * math.pi)
        p0 = centre + rr * (math.cos(ph) * e1 + math.sin(ph) * e2)
        iv = _clip_line_to_cylinder(p0, d, R, zlo, zhi)
        if iv is not None:
            break
    t0, t1 = iv
    track = _muon_segments(p0, d, R, zlo, zhi, 0)
    pos = t0 + rng.uniform(5.0, 50.0)
    cascades = []
    while pos < t1:
        cascades.append((pos, math.exp(rng.uniform(0.0, math.log(1e4)))))
        pos += rng.uniform(5.0, 50.0)
    cas = make_sources(len(cascades))
    for i, (t, _) in enumerate(cascades):
        q = p0 + t * d
        cas["x"][i], cas["y"][i], cas["z"][i] = q
    cas["dx"], cas["dy"], cas["dz"] = d[0], d[1], d[2]
    cas["type"] = SRC_CASCADE
    src = np.concatenate([track, cas])
    w = np.concatenate([track["length"].astype(np.float64),
                        np.array([e for _, e in cascades], np.float64)])
    n_total = int(round(math.exp(rng.uniform(math.log(photons_min), math.log(photons_max)))))
    share = np.floor(n_total * w / w.sum()).astype(np.int64)
    share[: n_total - int(share.sum())] += 1
    src["n_photons"] = share.astype(np.uint64)
    return src


def surrogate_sources(rng, n: int, photons: int, half_width: float = 450.0,
                      z_range: tuple = (-500.0, 500.0)) -> np.ndarray:
    """Light sources for the surrogate: 1 m Cherenkov segments at uniform
    positions in the instrumented volume, isotropic directions, `photons`
    photons each."""
    src = make_sources(n)
    src["x"] = rng.uniform(-half_width, half_width, n)
    src["y"] = rng.uniform(-half_width, half_width, n)
    src["z"] = rng.uniform(z_range[0], z_range[1], n)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    src["dx"], src["dy"], src["dz"] = d[:, 0], d[:, 1], d[:, 2]
    src["length"] = 1.0
    src["type"] = SRC_CHERENKOV
    src["n_photons"] = photons
    return src


def surrogate_sources_near(rng, n: int, photons: int, dom_xyz: np.ndarray,
                           r_near: float = 25.0, r_min: float = 0.5) -> np.ndarray:
    """Surrogate training sources close to DOMs, where direct light is bright
    and uniform placement rarely lands: each at a random DOM plus an offset
    uniform in the shell r_min <= |offset| <= r_near (segment midpoint),
    isotropic directions, 1 m Cherenkov segments."""
    src = make_sources(n)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = rng.normal(size=(n, 3))
    o /= np.linalg.norm(o, axis=1, keepdims=True)
    rad = np.cbrt(rng.uniform(r_min ** 3, r_near ** 3, n))
    centre = np.asarray(dom_xyz, np.float64)[rng.integers(0, len(dom_xyz), n)]
    start = centre + o * rad[:, None] - 0.5 * d     # the midpoint sits at the offset
    src["x"], src["y"], src["z"] = start[:, 0], start[:, 1], start[:, 2]
    src["dx"], src["dy"], src["dz"] = d[:, 0], d[:, 1], d[:, 2]
    src["length"] = 1.0
    src["type"] = SRC_CHERENKOV
    src["n_photons"] = photons
    return src
