"""Pins of the surrogate's oracle (CPU only): its analytic gradients against
central finite differences of its own loss (plain float64 network), the BF16
rounding against the binary32/BF16 bit layout, and the features against
hand-computed pairs."""
import math

import numpy as np
import pytest

from oracle import mlp as M
from paper_2405_05700_b300 import workloads as W


def _params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, 0.08 * scale, M.N_PARAMS)
    d = M.unpack(p)
    d["b5"] = -3.0
    return M.pack(d)


@pytest.mark.parametrize("act", ["silu", "hswish"])
def test_gradients_match_finite_differences(act):
    """For hard-swish W1 is scaled up so that the pre-activations of every
    layer spread over several units and each of its pieces (0, the quadratic,
    the identity) is exercised; the fraction in each piece is checked."""
    rng = np.random.default_rng(3)
    n = 48
    x = rng.normal(0, 1, (n, M.IN))
    nph = rng.uniform(50, 500, n)
    counts = rng.poisson(3.0, n).astype(np.float64)
    p = _params(4)
    if act == "hswish":
        d = M.unpack(p)
        d["W1"] = d["W1"] * 25.0
        p = M.pack(d)
        _, c = M.forward(p, x, nph, rounding=False, act=act)
        for z in c["z"]:
            assert (z < -3).mean() > 0.05 and (z > 3).mean() > 0.05
            assert (np.abs(z) < 3).mean() > 0.05
    loss, g = M.loss_and_grads(p, x, nph, counts, rounding=False, act=act)
    idx = np.concatenate([rng.choice(M.N_PARAMS - 1, 60, replace=False), [M.N_PARAMS - 1]])
    h = 1e-6
    for i in idx:
        e = np.zeros(M.N_PARAMS)
        e[i] = h
        lp, _ = M.loss_and_grads(p + e, x, nph, counts, rounding=False, act=act)
        lm, _ = M.loss_and_grads(p - e, x, nph, counts, rounding=False, act=act)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7, (i, fd, g[i])


def test_hard_swish_closed_form_values_and_slopes():
    """The definition's three pieces: 0 below -3, z^2/6 + z/2 between, z above
    (MobileNetV3's hard-swish), and its derivative z/3 + 1/2 inside, 0 and 1
    outside; the value is continuous at -3 and 3."""
    z = np.array([-10.0, -4.0, -3.0, -1.5, 0.0, 1.0, 2.5, 3.0, 4.0, 50.0])
    want = np.where(z <= -3, 0.0, np.where(z >= 3, z, z * z / 6 + z / 2))
    assert np.allclose(M.hswish(z), want, rtol=0, atol=1e-15)
    assert M.hswish(1.0) == pytest.approx(2.0 / 3.0) and M.hswish(-1.5) == pytest.approx(-0.375)
    slope = np.where(z <= -3, 0.0, np.where(z >= 3, 1.0, z / 3 + 0.5))
    assert np.allclose(M.hswish_grad(z), slope, rtol=0, atol=1e-15)
    # the derivative against central differences away from the kinks
    zz = np.linspace(-6, 6, 241)
    zz = zz[np.abs(np.abs(zz) - 3) > 1e-3]
    fd = (M.hswish(zz + 1e-6) - M.hswish(zz - 1e-6)) / 2e-6
    assert np.allclose(fd, M.hswish_grad(zz), atol=1e-6)
    for a, b in ((-3 - 1e-9, -3 + 1e-9), (3 - 1e-9, 3 + 1e-9)):
        assert abs(M.hswish(a) - M.hswish(b)) < 1e-8


def test_bf16_rounding_definition():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 0.0, 1e-40])
    r = M.bf16(x)
    assert r[0] == 1.0 and r[1] == 1.0               # tie to even (down)
    assert r[2] == 1.0 + 2 ** -7                     # exactly representable
    assert r[3] == 1.0 + 2 ** -6                     # tie to even (up)
    assert r[4] == -2.5 and r[5] == 0.0
    # every value has at most 8 significant bits
    y = M.bf16(np.random.default_rng(0).normal(size=1000))
    m, _ = np.frexp(y)
    assert np.all(m * 2 ** 8 == np.round(m * 2 ** 8))


def test_features_hand_computed():
    src = W.make_sources(2)
    src["x"], src["y"], src["z"] = [10.0, 0.0], [20.0, 0.0], [30.0, 0.0]
    src["dx"], src["dy"], src["dz"] = [0.0, 1.0], [0.0, 0.0], [1.0, 0.0]
    src["length"] = [2.0, 0.0]
    src["type"] = W.SRC_CHERENKOV
    doms = np.array([[10.0, 20.0, 61.0], [0.0, 5.0, 0.0]])
    b_e = np.array([0.01, 0.02, 0.03], np.float32).astype(np.float64)
    a = np.array([0.1, 0.2, 0.3], np.float32).astype(np.float64)
    f = M.features(src, [0, 1], [0, 1], doms, b_e, a, depth_top=1900.0, dz=10.0)
    tc = math.radians(41.0)
    # pair 0: midpoint (10, 20, 31), DOM 30 m straight above along the direction
    assert np.allclose(f[0, 0:3], [10 / 500, 20 / 500, 31 / 500])
    assert f[0, 3] == 0.0                                # polar angle 0
    assert np.allclose(f[0, 5:8], [0, 0, 0.3]) and np.isclose(f[0, 13], 0.3)
    assert np.isclose(f[0, 14], 1.0) and np.isclose(f[0, 15], math.log(31) / 5)
    # depth 1950 - 31 = 1919 -> layer 1 of the table starting at 1900 m
    assert np.isclose(f[0, 8], b_e[1] * 10) and np.isclose(f[0, 9], a[1] * 50)
    # on the axis: 41 degrees inside the cone, 30 sin(41 deg) m from its surface
    assert np.isclose(f[0, 16], -2 * tc) and np.isclose(f[0, 17], -3 * math.sin(tc))
    assert np.isclose(f[0, 18], math.exp(-15 * math.sin(tc)))
    # the DOM at height 61 m (depth 1889 m) lies above the table: layer 0
    assert np.isclose(f[0, 19], b_e[0] * 10) and np.isclose(f[0, 20], a[0] * 50)
    # the line spans layer coordinates -1.1 .. 1.9: 2.1 layers of row 0, 0.9 of row 1
    ma, mb = (2.1 * a[0] + 0.9 * a[1]) / 3.0, (2.1 * b_e[0] + 0.9 * b_e[1]) / 3.0
    assert np.isclose(f[0, 21], mb * 10) and np.isclose(f[0, 22], ma * 50)
    assert np.isclose(f[0, 23], 30 * ma) and np.isclose(f[0, 24], 3 * mb)
    assert np.allclose(f[0, 25:28], np.exp(-30 / np.array([10, 30, 100])))
    assert np.isclose(f[0, 28], 61 / 500) and np.isclose(f[0, 29], 1.0)
    assert np.isclose(f[0, 30], 1 / 7) and abs(f[0, 31]) < 1e-12
    # pair 1: direction +x, DOM 5 m along +y: perpendicular
    assert np.isclose(f[1, 3], 0.5) and np.isclose(f[1, 4], 0.0)
    assert np.isclose(f[1, 14], 0.0) and np.allclose(f[1, 10:13], [1, 0, 0])
    assert np.isclose(f[1, 16], 2 * (math.pi / 2 - tc))
    assert np.isclose(f[1, 17], 0.5 * math.sin(math.pi / 2 - tc))
    # depth 1950 -> layer 5, clamped to the last row, for the point, the DOM and the line
    assert np.isclose(f[1, 8], b_e[2] * 10) and np.isclose(f[1, 19], b_e[2] * 10)
    assert np.isclose(f[1, 21], b_e[2] * 10) and np.isclose(f[1, 22], a[2] * 50)
    assert np.isclose(f[1, 31], 0.05) and np.isclose(f[1, 30], 0.5)


def test_path_mean_against_numerical_integration():
    rng = np.random.default_rng(9)
    v = rng.uniform(0.01, 0.3, 12)
    u1 = rng.uniform(-3, 15, 200)
    u2 = rng.uniform(-3, 15, 200)
    got = M.path_mean(v, u1, u2)
    for a, b, g in zip(u1, u2, got):
        lo, hi = min(a, b), max(a, b)
        t = lo + (np.arange(200_000) + 0.5) * (hi - lo) / 200_000     # midpoint rule
        ref = v[np.clip(np.floor(t).astype(int), 0, len(v) - 1)].mean()
        assert abs(g - ref) <= 2e-4 * ref, (a, b, g, ref)
    # inside one layer: that layer's value; a homogeneous profile: its value
    assert np.allclose(M.path_mean(v, np.array([3.2]), np.array([3.9])), v[3])
    assert np.allclose(M.path_mean(np.full(5, 0.07), u1, u2), 0.07)


# ---- the network's definition, pinned against an independent float64 torch
# model built from the same parameters (torch.nn layers, torch's softplus and
# Poisson NLL, autograd), not against the oracle's own formulas ------------------

def _torch_net(params, act):
    import torch
    P = M.unpack(params)
    layers = []
    for l, (n_in, n_out) in enumerate(((M.IN, M.HID), (M.HID, M.HID), (M.HID, M.HID),
                                       (M.HID, M.HID)), start=1):
        lin = torch.nn.Linear(n_in, n_out, dtype=torch.float64)
        with torch.no_grad():
            lin.weight.copy_(torch.from_numpy(P[f"W{l}"]))
            lin.bias.copy_(torch.from_numpy(P[f"b{l}"]))
        layers += [lin, torch.nn.SiLU() if act == "silu" else torch.nn.Hardswish()]
    head = torch.nn.Linear(M.HID, 1, dtype=torch.float64)
    with torch.no_grad():
        head.weight.copy_(torch.from_numpy(P["w5"][None, :]))
        head.bias.fill_(float(P["b5"]))
    return torch.nn.Sequential(*layers, head)


def _torch_grads_in_oracle_layout(net):
    lin = [m for m in net if hasattr(m, "weight")]
    d = {}
    for l in (1, 2, 3, 4):
        d[f"W{l}"] = lin[l - 1].weight.grad.numpy()
        d[f"b{l}"] = lin[l - 1].bias.grad.numpy()
    d["w5"] = lin[4].weight.grad.numpy()[0]
    d["b5"] = float(lin[4].bias.grad.numpy()[0])
    return M.pack(d)


@pytest.mark.parametrize("act", ["silu", "hswish"])
def test_network_loss_and_gradients_match_torch(act):
    import torch
    rng = np.random.default_rng(11)
    n = 96
    x = rng.normal(0, 1, (n, M.IN))
    nph = rng.uniform(50, 500, n)
    counts = rng.poisson(3.0, n).astype(np.float64)
    counts[:8] = 0.0                                    # the n = 0 term of the loss
    p = _params(12, scale=3.0 if act == "hswish" else 1.0)
    net = _torch_net(p, act)
    xt = torch.from_numpy(x)
    lam_t = torch.from_numpy(nph) * torch.nn.functional.softplus(net(xt)[:, 0])
    # Poisson NLL with log input: exp(log lam) - n log lam = lam - n ln lam
    loss_t = torch.nn.functional.poisson_nll_loss(torch.log(lam_t), torch.from_numpy(counts),
                                                  log_input=True, full=False, reduction="mean")
    loss_t.backward()
    lam, _ = M.forward(p, x, nph, rounding=False, act=act)
    loss, g = M.loss_and_grads(p, x, nph, counts, rounding=False, act=act)
    assert np.allclose(lam, lam_t.detach().numpy(), rtol=1e-12, atol=0)
    assert loss == pytest.approx(float(loss_t), rel=1e-12)
    gt = _torch_grads_in_oracle_layout(net)
    scale = np.abs(gt).max()
    assert np.abs(g - gt).max() <= 1e-10 * scale


def test_rounded_forward_matches_torch_with_bf16_casts():
    """rounding=True: inputs, weights and hidden activations pass through BF16
    (torch's own float64 -> bfloat16 cast, round to nearest even)."""
    import torch
    rng = np.random.default_rng(13)
    x = rng.normal(0, 1, (64, M.IN))
    nph = rng.uniform(50, 500, 64)
    p = _params(14)
    P = M.unpack(p)

    def r(t):
        return t.to(torch.bfloat16).to(torch.float64)

    h = r(torch.from_numpy(x))
    for l in (1, 2, 3, 4):
        h = r(torch.nn.functional.silu(h @ r(torch.from_numpy(P[f"W{l}"])).T +
                                       torch.from_numpy(P[f"b{l}"])))
    lam_t = torch.from_numpy(nph) * torch.nn.functional.softplus(h @ torch.from_numpy(P["w5"]) +
                                                                 float(P["b5"]))
    lam, _ = M.forward(p, x, nph, rounding=True)
    assert np.allclose(lam, lam_t.numpy(), rtol=1e-12, atol=0)


# ---- Adam -----------------------------------------------------------------------

def test_adam_matches_torch_optimizer_over_several_steps():
    import torch
    rng = np.random.default_rng(15)
    n, lr = 1000, 3e-3
    p = rng.normal(0, 1, n)
    w = torch.nn.Parameter(torch.from_numpy(p.copy()))
    opt = torch.optim.Adam([w], lr=lr, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(n)
    v = np.zeros(n)
    for t in range(1, 8):
        g = rng.normal(0, 10.0 ** rng.uniform(-4, 1), n)
        w.grad = torch.from_numpy(g.copy())
        opt.step()
        p, m, v = M.adam_step(p, g, m, v, t, lr)
        st = opt.state[w]
        # torch forms the averages as m + (1 - b1)(g - m) (another rounding
        # order): compare at the averages' own scale
        assert np.abs(m - st["exp_avg"].numpy()).max() <= 1e-14 * np.abs(m).max()
        assert np.abs(v - st["exp_avg_sq"].numpy()).max() <= 1e-14 * np.abs(v).max()
        assert np.allclose(p, w.detach().numpy(), rtol=0, atol=1e-12)


def test_adam_first_step_and_scale_invariance():
    """From zero moments the bias corrections give m_hat = g and v_hat = g^2,
    so the first step is -lr g / (|g| + eps); with eps = 0 a step does not
    change when the gradient and the moments are scaled by c and c^2."""
    rng = np.random.default_rng(16)
    g = rng.normal(0, 1, 500) * 10.0 ** rng.uniform(-6, 2, 500)
    p0 = rng.normal(0, 1, 500)
    p1, m1, v1 = M.adam_step(p0, g, np.zeros(500), np.zeros(500), 1, 0.01)
    assert np.allclose(p1 - p0, -0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m1, 0.1 * g, rtol=1e-15) and np.allclose(v1, 0.001 * g * g, rtol=1e-15)
    m0, v0 = rng.normal(0, 1, 500), rng.uniform(0.5, 2, 500)
    a = M.adam_step(p0, g, m0, v0, 5, 0.01, eps=0.0)[0]
    b = M.adam_step(p0, 7.0 * g, 7.0 * m0, 49.0 * v0, 5, 0.01, eps=0.0)[0]
    assert np.allclose(a, b, rtol=0, atol=1e-13)
