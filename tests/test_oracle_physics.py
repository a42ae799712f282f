"""Pins of the whole oracle propagation against closed forms and invariants
(CPU only).

* No scattering, homogeneous absorption, one DOM: the hit fraction equals the
  solid-angle integral of the survival probability (exact quadrature).
* The same with layered absorption and the DOM in other layers: the optical
  depth along each ray comes from an independent fine-grid integral.
* No DOMs, no scattering: the escape fraction equals the direction average of
  exp(-a * exit distance) (bisection for the exit distance).
* Infinite homogeneous medium: every photon is absorbed, the path is Exp(a),
  the scatter count has mean b/a, and the mean cosine between successive
  directions is g.
* Conservation: hits + absorbed + escaped = emitted, exactly.
* Births: Cherenkov photons leave at 41 degrees to the track; point sources
  emit isotropically.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2405_05700_b300 import workloads as W


def _one_dom(d_below, r):
    return W.Geometry(np.array([[0.0, 0.0, -d_below]], np.float32), np.zeros(1, np.int32), r)


def _binomial_z(k, n, p):
    return (k - n * p) / math.sqrt(n * p * (1 - p))


@pytest.mark.parametrize("a", [0.01, 0.0])
def test_no_scatter_single_dom_hit_fraction(orc, a):
    d, r = 10.0, 1.0
    geom = _one_dom(d, r)
    ice = W.ice_homogeneous(0.0, a, g=0.9, n_layers=1, depth_top=0.0)
    m = orc.Model(geom, ice, seed=17, world_margin=1000.0)
    N = 4_000_000
    hits, counts, _ = orc.propagate(m, W.single_event(W.point_source(0, 0, 0, N), 3))
    mu0 = math.sqrt(1 - r * r / (d * d))
    a32 = float(np.float32(a))

    def surv(mu):
        t = d * mu - math.sqrt(max(0.0, r * r - d * d * (1 - mu * mu)))
        return math.exp(-a32 * t)

    P = 0.5 * integrate.quad(surv, mu0, 1.0, epsabs=1e-14, epsrel=1e-12)[0]
    if a == 0.0:
        assert P == pytest.approx((1 - mu0) / 2, rel=1e-10)
        assert counts[0, 0] == 0           # nothing is absorbed without absorption
    k = int(hits[0, 0])
    assert abs(_binomial_z(k, N, P)) < 4, (k, N * P)
    assert int(hits.sum() + counts[0, 0] + counts[0, 1]) == N


def test_no_scatter_layered_absorption_hit_fraction(orc):
    # source in the middle of a layer, DOM 25 m below it (three layers away),
    # absorption different in every layer
    L = 20
    ice = W.Ice(np.zeros(L, np.float32), (0.004 + 0.003 * np.arange(L)).astype(np.float32),
                1900.0, 10.0, 0.9)
    z_src = 1950.0 - 1955.0            # depth 1955: middle of layer 5
    d, r = 25.0, 1.5
    geom = W.Geometry(np.array([[0.0, 0.0, z_src - d]], np.float32), np.zeros(1, np.int32), r)
    m = orc.Model(geom, ice, seed=5, world_margin=500.0)
    N = 4_000_000
    hits, counts, _ = orc.propagate(m, W.single_event(W.point_source(0, 0, z_src, N), 1))
    a = ice.a.astype(np.float64)

    mu0 = math.sqrt(1 - r * r / (d * d))
    # Gauss-Legendre nodes in mu on [mu0, 1]; the ray at angle acos(mu) to
    # the downward axis enters the sphere at distance t and gains depth t*mu;
    # its optical depth by the midpoint rule on a fine grid along the ray.
    x, wx = np.polynomial.legendre.leggauss(3000)
    mu = mu0 + (x + 1) * (1 - mu0) / 2
    t = d * mu - np.sqrt(np.maximum(0.0, r * r - d * d * (1 - mu * mu)))
    n = 4000
    s = (np.arange(n)[None, :] + 0.5) * (t[:, None] / n)
    depth = 1955.0 + s * mu[:, None]
    i = np.clip(np.floor((depth - 1900.0) / 10.0).astype(int), 0, L - 1)
    tau = a[i].sum(1) * (t / n)
    P = 0.5 * float((wx * np.exp(-tau)).sum()) * (1 - mu0) / 2
    k = int(hits[0, 0])
    assert abs(_binomial_z(k, N, P)) < 4, (k, N * P)


def test_no_scatter_escape_fraction(orc):
    geom = W.Geometry(np.zeros((0, 3), np.float32), np.zeros(0, np.int32), 0.1651)
    a = 0.02
    ice = W.ice_homogeneous(0.0, a, n_layers=1)
    M = 60.0                            # world: radius 60, z in [-60, 60]
    m = orc.Model(geom, ice, seed=8, world_margin=M)
    p0 = np.array([10.0, -5.0, 20.0])
    N = 2_000_000
    hits, counts, _ = orc.propagate(m, W.single_event(W.point_source(*p0, N), 0))
    esc = int(counts[0, 1])
    # direction average of exp(-a t_exit): Gauss-Legendre in mu, periodic in phi
    nm, nphi = 1500, 1500
    mu, wmu = np.polynomial.legendre.leggauss(nm)
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    MU, PHI = np.meshgrid(mu, phi, indexing="ij")
    st = np.sqrt(1 - MU ** 2)
    D = np.stack([st * np.cos(PHI), st * np.sin(PHI), MU], -1).reshape(-1, 3)
    lo, hi = np.zeros(D.shape[0]), np.full(D.shape[0], 400.0)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        q = p0 + mid[:, None] * D
        ins = (q[:, 0] ** 2 + q[:, 1] ** 2 <= M * M) & (np.abs(q[:, 2]) <= M)
        lo, hi = np.where(ins, mid, lo), np.where(ins, hi, mid)
    f = np.exp(-float(np.float32(a)) * lo).reshape(nm, nphi).mean(1)
    P = 0.5 * float((wmu * f).sum())
    assert abs(_binomial_z(esc, N, P)) < 4, (esc, N * P)
    assert int(counts[0, 0] + esc) == N and hits.size == 0


def test_infinite_homogeneous_medium(orc):
    geom = W.Geometry(np.zeros((0, 3), np.float32), np.zeros(0, np.int32), 0.1651)
    be, a, g = 0.05, 0.01, 0.9
    ice = W.ice_homogeneous(be, a, g=g, n_layers=3, depth_top=1900.0)
    m = orc.Model(geom, ice, seed=2, world_margin=1e5)
    N = 40000
    _, counts, st = orc.propagate(m, W.single_event(W.point_source(0, 0, 0, N), 4))
    assert int(counts[0, 0]) == N and int(counts[0, 1]) == 0 and int(counts[0, 2]) == 0
    a32 = float(np.float32(a))
    b32 = float(np.float32(be)) / (1 - g)
    mean_path = st["path"] / N
    assert abs(mean_path - 1 / a32) < 4 * (1 / a32) / math.sqrt(N)
    m_sc = b32 / a32
    mean_sc = st["scatters"] / N
    assert abs(mean_sc - m_sc) < 4 * math.sqrt(m_sc * (1 + m_sc) / N)
    assert abs(st["cos_sum"] / st["scatters"] - g) < 1e-3
    # steps = scatters + one final step per photon
    assert int(counts[0, 3]) == int(st["scatters"]) + N


def test_conservation_tiny_config(orc):
    geom, ice = W.geometry_tiny(), W.ice_tiny()
    m = orc.Model(geom, ice, seed=0)
    b = W.sources_tiny(200_000)
    hits, counts, _ = orc.propagate(m, b)
    assert int(hits.sum() + counts[0, 0] + counts[0, 1]) == 200_000
    assert int(counts[0, 2]) == 0


def test_conservation_muon_bundles_and_step_cap(orc):
    geom = W.geometry_full()
    ice = W.ice_full()
    b = W.events_full(n_events=12, seed=3)
    for max_steps in (100_000, 7):
        m = orc.Model(geom, ice, seed=1, max_steps=max_steps)
        hits, counts, _ = orc.propagate(m, b)
        emitted = b.photons_per_event().astype(np.int64)
        got = hits.sum(1).astype(np.int64) + counts[:, 0].astype(np.int64) + counts[:, 1].astype(np.int64)
        assert np.array_equal(got, emitted)
        if max_steps == 7:
            assert counts[:, 2].sum() > 0 and np.all(counts[:, 2] <= counts[:, 0])
        else:
            assert counts[:, 2].sum() == 0


def test_cherenkov_birth_angle_and_position(orc):
    geom, ice = W.geometry_tiny(), W.ice_tiny()
    m = orc.Model(geom, ice, seed=9)
    src = W.make_sources(1)
    d = np.array([0.3, -0.2, -0.9])
    d /= np.linalg.norm(d)
    src["x"], src["y"], src["z"] = 5.0, 6.0, 7.0
    src["dx"], src["dy"], src["dz"] = d
    src["length"] = 1.0
    src["type"] = W.SRC_CHERENKOV
    src["n_photons"] = 20000
    d32 = np.array([src["dx"][0], src["dy"][0], src["dz"][0]], np.float64)
    d32 /= np.linalg.norm(d32)
    _, _, birth, _ = orc.trace(m, 0, src, np.arange(20000), n_trace=1)
    cosang = birth[:, 3:] @ d32
    assert np.max(np.abs(cosang - math.cos(math.radians(41.0)))) < 1e-12
    t = (birth[:, :3] - [5.0, 6.0, 7.0]) @ d32
    assert t.min() >= 0 and t.max() <= 1.0 + 1e-6
    assert abs(t.mean() - 0.5) < 4 * math.sqrt(1 / 12 / 20000)
    off = birth[:, :3] - [5.0, 6.0, 7.0] - t[:, None] * d32
    assert np.max(np.linalg.norm(off, axis=1)) < 1e-5   # births lie on the segment
    # azimuth about the track is uniform: the transverse part averages to zero
    perp = birth[:, 3:] - cosang[:, None] * d32
    assert np.all(np.abs(perp.mean(0)) < 4 * math.sin(math.radians(41)) / math.sqrt(2 * 20000))


def test_point_source_birth_is_isotropic(orc):
    m = orc.Model(W.geometry_tiny(), W.ice_tiny(), seed=10)
    n = 100000
    _, _, birth, _ = orc.trace(m, 2, W.point_source(1, 2, 3, n), np.arange(n), n_trace=1)
    assert np.allclose(birth[:, :3], [1, 2, 3])
    dirs = birth[:, 3:]
    assert np.max(np.abs(np.linalg.norm(dirs, axis=1) - 1)) < 1e-12
    assert np.all(np.abs(dirs.mean(0)) < 4 * math.sqrt(1 / 3 / n))
    assert abs((dirs[:, 2] ** 2).mean() - 1 / 3) < 4 * math.sqrt(4 / 45 / n)


def test_trace_agrees_with_propagate(orc):
    # per-photon outcomes summed over an event equal the event's tallies
    geom, ice = W.geometry_tiny(), W.ice_tiny()
    m = orc.Model(geom, ice, seed=4)
    b = W.sources_tiny(30000)
    hits, counts, _ = orc.propagate(m, b)
    out, ns, _, tr = orc.trace(m, 0, b.sources, np.arange(30000), n_trace=10)
    assert np.array_equal(np.bincount(out[out >= 0], minlength=geom.n_dom), hits[0])
    assert int((out == -1).sum()) == int(counts[0, 0])
    assert int((out == -2).sum()) == int(counts[0, 1])
    assert int(ns.sum()) == int(counts[0, 3])
    # trace rows are filled exactly up to the number of scatters
    filled = np.isfinite(tr[:, :, 0]).sum(1)
    assert np.array_equal(filled, np.minimum(ns - 1, 10))
