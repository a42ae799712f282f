"""Pins of the oracle's scattering step (CPU only): the Henyey-Greenstein
sampler against the closed-form HG distribution, and the direction rotation
against the geometry it must satisfy."""
import numpy as np


def hg_cdf(mu, g):
    """P(cos theta <= mu) for the Henyey-Greenstein phase function (closed
    form of the integral of (1 - g^2) / (2 (1 + g^2 - 2 g mu)^{3/2}))."""
    return (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))


def test_hg_inverts_the_closed_form_cdf(orc):
    u = (np.arange(1, 200000, 2, dtype=np.float64)) / 200000.0
    for g in (0.9, 0.5, 0.1, -0.3):
        mu = orc.hg(g, u)
        assert np.all(np.abs(mu) <= 1.0)
        assert np.max(np.abs(hg_cdf(mu, g) - u)) < 1e-9
        assert np.all(np.diff(mu) > 0)  # monotone in u


def test_hg_moments(orc):
    # <mu> = g and <P2(mu)> = g^2 for the HG phase function; Philox draws.
    n = 1 << 21
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    ctr[:, 2] = 1
    u = orc.u01(orc.philox(ctr, np.array([3, 4], np.uint32))[:, 1])
    g = 0.9
    mu = orc.hg(g, u)
    assert abs(mu.mean() - g) < 1e-3
    p2 = 0.5 * (3 * mu * mu - 1)
    assert abs(p2.mean() - g * g) < 4 * p2.std() / np.sqrt(n)
    iso = orc.hg(0.0, u)
    assert abs(iso.mean()) < 4 * np.sqrt(1 / 3 / n)
    assert abs((iso ** 2).mean() - 1 / 3) < 4 * np.sqrt(4 / 45 / n)


def _random_dirs(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def test_rotation_keeps_polar_angle_and_unit_length(orc):
    rng = np.random.default_rng(5)
    n = 100000
    d = _random_dirs(rng, n)
    d[:50, :] = [0, 0, 1]     # the pole branch
    d[50:100, :] = [0, 0, -1]
    mu = rng.uniform(-1, 1, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    out = orc.rotate(d, mu, phi)
    assert np.max(np.abs(np.linalg.norm(out, axis=1) - 1)) < 1e-12
    cosang = (d * out).sum(1)
    general = np.abs(d[:, 2]) <= 0.99999
    assert np.max(np.abs(cosang[general] - mu[general])) < 1e-10
    assert np.max(np.abs(cosang[~general] - mu[~general])) < 1e-4


def test_rotation_azimuth_is_a_rotation_about_d(orc):
    """For fixed d and mu, the new direction moves on the cone about d and the
    azimuth parameter is the angle along it: directions at phi and phi + dphi
    make the angle dphi when projected on the plane normal to d."""
    rng = np.random.default_rng(6)
    n = 20000
    d = _random_dirs(rng, n)
    d = d[np.abs(d[:, 2]) <= 0.99]
    n = d.shape[0]
    mu = rng.uniform(-0.95, 0.95, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    dphi = rng.uniform(0.1, 3.0, n)
    a = orc.rotate(d, mu, phi)
    b = orc.rotate(d, mu, phi + dphi)
    pa = a - (a * d).sum(1, keepdims=True) * d
    pb = b - (b * d).sum(1, keepdims=True) * d
    c = (pa * pb).sum(1) / (np.linalg.norm(pa, axis=1) * np.linalg.norm(pb, axis=1))
    assert np.max(np.abs(c - np.cos(dphi))) < 1e-9
    # and the sense of rotation is the same for every d (right-handed about d)
    s = (np.cross(pa, pb) * d).sum(1)
    assert np.all(np.sign(s) == np.sign(np.sin(dphi)))


def test_isotropic_rotation_is_isotropic(orc):
    # mu uniform in [-1, 1] and phi uniform: new directions uniform on the
    # sphere whatever d is.
    rng = np.random.default_rng(7)
    n = 400000
    d = np.tile([[0.3, -0.5, 0.812403840463596]], (n, 1))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out = orc.rotate(d, rng.uniform(-1, 1, n), rng.uniform(0, 2 * np.pi, n))
    m = out.mean(0)
    assert np.all(np.abs(m) < 4 * np.sqrt(1 / 3 / n))
    cov = out.T @ out / n
    assert np.max(np.abs(cov - np.eye(3) / 3)) < 4 * np.sqrt(4 / 45 / n) + 2e-3
