"""Pins of the oracle's geometric pieces (CPU only): the layer walk against an
independent optical-depth integral, the world exit against bisection, and the
first-DOM test against brute force and against point-to-segment distances."""
import numpy as np
import pytest

from paper_2405_05700_b300 import workloads as W


def _model(orc, geom=None, ice=None, **kw):
    geom = geom if geom is not None else W.geometry_tiny()
    ice = ice if ice is not None else W.ice_tiny()
    return orc.Model(geom, ice, **kw)


def _cum_tau(ice, coeff, z_grid, z0_depth=1950.0):
    """Optical depth from z_grid[0] along z_grid (monotone) by the midpoint
    rule on a fine grid -- independent of the oracle's boundary walk."""
    zm = 0.5 * (z_grid[1:] + z_grid[:-1])
    depth = z0_depth - zm
    i = np.clip(np.floor((depth - ice.depth_top) / ice.dz).astype(int), 0, ice.n_layers - 1)
    dtau = coeff[i] * np.abs(np.diff(z_grid))
    return np.concatenate([[0.0], np.cumsum(dtau)])


@pytest.mark.parametrize("w", [-1.0, 1.0, -0.37, 0.61])
def test_walk_absorption_length_matches_optical_depth_integral(orc, w):
    ice = W.ice_tiny()
    ice.b_e[:] = 0.0                       # no scattering: the step ends by absorption
    m = _model(orc, ice=ice)
    rng = np.random.default_rng(11)
    z0 = rng.uniform(-450, 450, 200)
    tau_a = rng.uniform(0.01, 3.0, 200)
    S, absorbed, _, _ = orc.walk(m, z0, w, 1e30, tau_a)
    assert np.all(absorbed)
    a = ice.a.astype(np.float64)
    for zi, ta, s in zip(z0, tau_a, S):
        # fine grid in z along the direction of travel; exact layer edges are
        # included so that the midpoint rule is exact per cell
        span = 3.0 / 0.005 + 20.0
        zs = np.sort(np.concatenate([np.linspace(zi, zi + np.sign(w) * span, 200001),
                                     1950.0 - ice.depth_top - ice.dz * np.arange(ice.n_layers + 1)]))
        zs = zs[(zs - zi) * np.sign(w) >= 0]
        if w < 0:
            zs = zs[::-1]
        tau = _cum_tau(ice, a, zs)
        # optical depth along the path is the vertical integral over |w|
        dz_needed = np.interp(ta * abs(w), tau, np.abs(zs - zi))
        assert abs(s * abs(w) - dz_needed) < 1e-6 * max(1.0, dz_needed)


def test_walk_homogeneous_is_min_of_two_exponentials(orc):
    ice = W.ice_homogeneous(0.05, 0.01, g=0.9, n_layers=5, depth_top=1000.0)
    m = _model(orc, ice=ice)
    rng = np.random.default_rng(3)
    n = 1000
    ts, ta = rng.exponential(size=n), rng.exponential(size=n)
    w = rng.uniform(-1, 1, n)
    S, ab, _, ta_end = orc.walk(m, rng.uniform(-500, 500, n), w, ts, ta)
    # the tables arrive as float32; the oracle widens them
    b = float(np.float32(0.05)) / (1 - 0.9)
    a = float(np.float32(0.01))
    exp_S = np.minimum(ts / b, ta / a)
    assert np.allclose(S, exp_S, rtol=1e-12, atol=1e-12)
    assert np.array_equal(ab, ta / a <= ts / b)
    assert np.allclose(ta_end[~ab], ta[~ab] - a * S[~ab], atol=1e-12)


def test_walk_effective_vs_geometric_scattering_flag(orc):
    ice = W.ice_homogeneous(0.05, 1e-9, g=0.9, n_layers=1, depth_top=1000.0)
    S_eff = orc.walk(_model(orc, ice=ice), [0.0], 1.0, 1.0, 50.0)[0][0]
    S_geo = orc.walk(_model(orc, ice=ice, scatter_coeff_is_effective=False), [0.0], 1.0, 1.0, 50.0)[0][0]
    assert abs(S_eff - 1.0 / 0.5) < 1e-7 and abs(S_geo - 1.0 / 0.05) < 1e-6


def test_layer_at_rules(orc):
    m = _model(orc)  # 100 layers from depth 1450: layer i spans z in (500-10(i+1), 500-10 i]
    z = np.array([500.0, 500.0, 495.0, 490.0, 490.0, 490.0, -499.9, 600.0, -600.0])
    w = np.array([-1.0, 1.0, 1.0, -0.5, 0.5, 0.0, 1.0, -1.0, 1.0])
    assert list(orc.layer_at(m, z, w)) == [0, 0, 0, 1, 0, 1, 99, 0, 99]


def test_world_exit_matches_bisection(orc):
    m = _model(orc)
    R, zlo, zhi = orc.world(m)
    assert R == pytest.approx(125.0 + 100.0) and zlo == pytest.approx(-503.0 - 100.0)
    rng = np.random.default_rng(9)
    n = 2000
    r = R * np.sqrt(rng.uniform(0, 1, n))
    ang = rng.uniform(0, 2 * np.pi, n)
    p = np.stack([r * np.cos(ang), r * np.sin(ang), rng.uniform(zlo, zhi, n)], 1)
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t = orc.world_exit(m, p, d)

    def inside(q):
        return (q[:, 0] ** 2 + q[:, 1] ** 2 <= R * R) & (q[:, 2] >= zlo) & (q[:, 2] <= zhi)

    lo, hi = np.zeros(n), np.full(n, 4 * R + (zhi - zlo))
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        ins = inside(p + mid[:, None] * d)
        lo = np.where(ins, mid, lo)
        hi = np.where(ins, hi, mid)
    assert np.max(np.abs(t - lo)) < 1e-7
    # a point outside leaves at once
    assert orc.world_exit(m, [[R + 1, 0, 0]], [[-1, 0, 0]])[0] == 0.0


def _random_segments_near_doms(rng, geom, n, reach=3.0):
    k = rng.integers(0, geom.n_dom, n)
    c = geom.xyz[k].astype(np.float64)
    p = c + rng.uniform(-reach, reach, (n, 3))
    d = rng.normal(size=(n, 3))
    aim = slice(n // 10, n // 2)        # aimed near the DOM: grazing and direct hits
    d[aim] = c[aim] - p[aim] + rng.normal(0.0, 0.15, (n // 2 - n // 10, 3))
    d[: n // 10, :2] *= 1e-4            # near-vertical steps along the strings
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    S = rng.exponential(2.0, n)
    S[: n // 20] = rng.uniform(20, 200, n // 20)   # long steps crossing several DOMs
    return p, d, S


def test_first_hit_bbox_filter_equals_brute_force(orc):
    geom = W.geometry_tiny()
    rng = np.random.default_rng(21)
    p, d, S = _random_segments_near_doms(rng, geom, 200000)
    dom_f, t_f = orc.first_hit(_model(orc, geom=geom), p, d, S)
    dom_b, t_b = orc.first_hit(_model(orc, geom=geom, brute_force=True), p, d, S)
    assert np.array_equal(dom_f, dom_b)
    hit = dom_b >= 0
    assert np.array_equal(t_f[hit], t_b[hit])
    assert hit.mean() > 0.01


def test_first_hit_geometry(orc):
    """Independent of the quadratic: a segment meets a sphere iff its closest
    point is within r; the reported point lies on the sphere (or the start is
    inside), and no sphere is met earlier (probing just before t)."""
    geom = W.geometry_tiny()
    m = _model(orc, geom=geom, brute_force=True)
    rng = np.random.default_rng(22)
    n = 50000
    p, d, S = _random_segments_near_doms(rng, geom, n, reach=1.0)
    dom, t = orc.first_hit(m, p, d, S)
    c = geom.xyz.astype(np.float64)
    r = geom.dom_radius
    # closest-approach distance of each segment to every DOM centre
    hit_any = np.zeros(n, bool)
    margin = np.full(n, np.inf)
    for k in range(geom.n_dom):
        v = c[k] - p
        s = np.clip((v * d).sum(1), 0.0, S)
        dist = np.linalg.norm(p + s[:, None] * d - c[k], axis=1)
        hit_any |= dist <= r
        margin = np.minimum(margin, np.abs(dist - r))
    clear = margin > 1e-9
    assert np.array_equal((dom >= 0)[clear], hit_any[clear])
    h = np.nonzero(dom >= 0)[0]
    q = p[h] + t[h, None] * d[h]
    rad = np.linalg.norm(q - c[dom[h]], axis=1)
    inside0 = np.linalg.norm(p[h] - c[dom[h]], axis=1) <= r
    assert np.all(np.abs(rad[~inside0] - r) < 1e-9)
    assert np.all(t[h][inside0] == 0.0)
    # nothing earlier: the point a little before t is outside every sphere
    early = h[t[h] > 1e-6]
    qe = p[early] + (t[early] - 1e-6)[:, None] * d[early]
    dmin = np.min(np.linalg.norm(qe[:, None, :] - c[None, :, :], axis=2), axis=1)
    assert np.all(dmin > r)
