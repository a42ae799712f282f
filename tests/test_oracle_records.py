"""Pins of the oracle's compact hit records (CPU only).

* No scattering, no absorption, one DOM: every hit time is the straight
  path to the sphere's near side at the group velocity, so it lies in
  [n_g (d - r) / c, n_g sqrt(d^2 - r^2) / c], and the mean over hits equals
  the solid-angle average of that distance over the DOM's cone (quadrature).
* A Cherenkov segment: each time lies between the bounds set by the
  emission offset along the segment (at c) and the distance from the
  emission point to the sphere.
* The records' DOM histogram equals the per-DOM hits of the propagation of
  the same event, exactly.
* Acceptance weights: with a DOM straight below (above) a point source and no
  scattering, every hitting photon moves down (up) within the DOM's small
  cone, so each weight lies within the polynomial's range over that cone;
  constant polynomials above 1 or below 0 clamp to 1 and 0.
"""
import math

import numpy as np
from scipy import integrate

from paper_2405_05700_b300 import workloads as W

C_M_PER_NS = 0.299792458


def _one_dom(centre, r):
    return W.Geometry(np.array([centre], np.float32), np.zeros(1, np.int32), r)


def test_no_scatter_point_source_hit_times(orc):
    d, r, ng = 10.0, 1.0, 1.35
    geom = _one_dom([0.0, 0.0, -d], r)
    ice = W.ice_homogeneous(0.0, 0.0, g=0.9, n_layers=1, depth_top=0.0)
    m = orc.Model(geom, ice, seed=5, world_margin=1000.0)
    rec = orc.hit_records(m, 2, W.point_source(0, 0, 0, 400_000), group_index=ng)
    assert rec["n"] > 500 and np.all(rec["dom"] == 0) and np.all(rec["source"] == 0)
    path = rec["time_ns"] * C_M_PER_NS / ng
    f32 = 1e-4                       # the DOM centre and radius are binary32 values
    assert path.min() >= d - r - f32 and path.max() <= math.sqrt(d * d - r * r) + f32
    mu0 = math.sqrt(1 - r * r / (d * d))

    def near_side(mu):
        return d * mu - math.sqrt(max(0.0, r * r - d * d * (1 - mu * mu)))

    mean = integrate.quad(near_side, mu0, 1.0, epsabs=1e-13)[0] / (1 - mu0)
    sd = path.std()
    assert abs(path.mean() - mean) < 4 * sd / math.sqrt(len(path)), (path.mean(), mean)


def test_cherenkov_segment_hit_time_bounds(orc):
    r, ng, L = 0.5, 1.35, 20.0
    centre = np.array([6.0, 0.0, 10.0])
    geom = _one_dom(centre, r)
    ice = W.ice_homogeneous(0.0, 0.0, g=0.9, n_layers=1, depth_top=0.0)
    m = orc.Model(geom, ice, seed=9, world_margin=1000.0)
    src = W.make_sources(1)
    src["dx"], src["dy"], src["dz"] = 0.0, 0.0, 1.0
    src["length"] = L
    src["type"] = W.SRC_CHERENKOV
    src["n_photons"] = 2_000_000
    rec = orc.hit_records(m, 4, src, group_index=ng)
    assert rec["n"] > 200
    # emission at height t0 in [0, L]: c t = t0 + n_g * path, |path - dist(t0)| <= r
    t0 = np.linspace(0.0, L, 20001)
    dist = np.sqrt(centre[0] ** 2 + (centre[2] - t0) ** 2)
    lo, hi = np.min(t0 + ng * (dist - r)), np.max(t0 + ng * (dist + r))
    ct = rec["time_ns"] * C_M_PER_NS
    assert ct.min() >= lo - 1e-3 and ct.max() <= hi + 1e-3


def test_record_histogram_equals_propagated_hits(orc):
    geom, ice = W.geometry_tiny(), W.ice_tiny()
    m = orc.Model(geom, ice, seed=0)
    src = np.concatenate([W.point_source(0.0, 0.0, 0.0, 30_000),
                          W.point_source(60.0, 20.0, -100.0, 30_000)])
    rec = orc.hit_records(m, 3, src)
    hits, counts, _ = orc.propagate(m, W.single_event(src, 3))
    assert rec["n"] == int(hits.sum())
    assert np.array_equal(np.bincount(rec["dom"], minlength=geom.n_dom), hits[0])
    assert set(np.unique(rec["source"])) <= {0, 1}
    assert np.all(rec["time_ns"] > 0)


def test_acceptance_weights_follow_the_incidence_direction(orc):
    d, r = 10.0, 1.0
    ice = W.ice_homogeneous(0.0, 0.0, g=0.9, n_layers=1, depth_top=0.0)
    acc = [0.25, 0.5, 0.25]                      # 0.25 (1 + eta)^2

    def poly(eta):
        return 0.25 * (1.0 + eta) ** 2

    eta_min = math.sqrt(1 - r * r / (d * d))    # the cone's edge: |eta| >= cos of its half-angle
    for zc, lo, hi in ((-d, poly(-1.0), poly(-eta_min)), (d, poly(eta_min), poly(1.0))):
        m = orc.Model(_one_dom([0.0, 0.0, zc], r), ice, seed=3, world_margin=1000.0)
        rec = orc.hit_records(m, 1, W.point_source(0, 0, 0, 200_000), acceptance=acc)
        assert rec["n"] > 200
        w = rec["weight"]
        assert w.min() >= lo - 1e-12 and w.max() <= hi + 1e-12, (zc, w.min(), w.max(), lo, hi)
    m = orc.Model(_one_dom([0.0, 0.0, -d], r), ice, seed=3, world_margin=1000.0)
    src = W.point_source(0, 0, 0, 50_000)
    assert np.all(orc.hit_records(m, 1, src)["weight"] == 1.0)
    assert np.all(orc.hit_records(m, 1, src, acceptance=[2.0])["weight"] == 1.0)
    assert np.all(orc.hit_records(m, 1, src, acceptance=[-0.5])["weight"] == 0.0)
