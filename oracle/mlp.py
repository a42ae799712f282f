"""Oracle of the learned surrogate: the MLP's features, forward pass, loss and
gradients, written out plainly in numpy float64.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's checks); it does
not import the CUDA library.

The network (the surrogate has no counterpart in the paper; it is a BF16
multilayer perceptron with FP32 accumulation whose output is a Poisson mean):
    h1 = act(W1 x + b1), h_l = act(W_l h_{l-1} + b_l) (l = 2..4),
    z = w5 . h4 + b5,  lambda = n_photons * softplus(z),
    loss = mean over pairs of (lambda - n ln lambda),
with act = silu(z) = z / (1 + exp(-z)), or hard-swish
    hswish(z) = z * clamp(z / 6 + 1/2, 0, 1)
(Howard et al., "Searching for MobileNetV3", 2019), whose derivative is taken
as t + z / 6 inside (-3, 3) and t outside, t = clamp(z / 6 + 1/2, 0, 1).
With rounding=True the values the device stores in BF16 are rounded to BF16
at the same points (weights W1..W4, inputs, hidden activations, the stored
pre-activations used by the backward pass, and the back-propagated dL/dz of
each layer); everything else is float64.  With rounding=False it is the plain
float64 network, which the finite-difference pin checks.
The optimizer is Adam (adam_step).
"""
from __future__ import annotations

import math

import numpy as np

HID, IN = 256, 32
N_PARAMS = HID * IN + HID + 3 * (HID * HID + HID) + HID + 1


def bf16(x):
    """Nearest BF16 value of each element (via binary32, ties to even)."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    r = ((u >> 16) & 1) + 0x7FFF
    return (((u + r) >> 16) << 16).astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = {}
    out["W1"] = p[o:o + HID * IN].reshape(HID, IN); o += HID * IN
    out["b1"] = p[o:o + HID]; o += HID
    for l in (2, 3, 4):
        out[f"W{l}"] = p[o:o + HID * HID].reshape(HID, HID); o += HID * HID
        out[f"b{l}"] = p[o:o + HID]; o += HID
    out["w5"] = p[o:o + HID]; o += HID
    out["b5"] = p[o]; o += 1
    assert o == N_PARAMS
    return out


def pack(d):
    parts = [d["W1"].ravel(), d["b1"]]
    for l in (2, 3, 4):
        parts += [d[f"W{l}"].ravel(), d[f"b{l}"]]
    parts += [d["w5"], np.array([d["b5"]])]
    return np.concatenate(parts)


def _layer_index(u, L):
    return np.clip(np.floor(u).astype(np.int64), 0, L - 1)


def path_mean(v, u1, u2):
    """Mean of the piecewise-constant profile v (one value per layer, the
    edge layers extended outward) over the layer coordinate interval
    [u1, u2] (either order): the exact integral divided by the length, the
    layer's own value when both ends fall in one layer."""
    v = np.asarray(v, np.float64)
    L = len(v)
    cum = np.concatenate([[0.0], np.cumsum(v)])[:L]          # sum of the layers before i
    i1, i2 = _layer_index(u1, L), _layer_index(u2, L)
    F1 = cum[i1] + (u1 - i1) * v[i1]
    F2 = cum[i2] + (u2 - i2) * v[i2]
    same = i1 == i2
    du = np.where(same, 1.0, u2 - u1)
    return np.where(same, v[i1], ((cum[i2] - cum[i1]) + (u2 - i2) * v[i2] - (u1 - i1) * v[i1]) / du)


def features(sources, pair_src, pair_dom, dom_xyz, b_e, a, depth_top, dz, depth_of_z0=1950.0,
             theta_c=math.radians(41.0)):
    """The IN = 32 inputs of each (source, DOM) pair, float64, unrounded.

    p = segment midpoint, d = unit direction, e = DOM - p, r = |e|,
    c = d.e / max(r, 1 mm), delta = acos(c) - theta_c (angle from the
    Cherenkov cone), rho = r sin(delta) (distance from the cone's surface),
    u = (z_top - z) / dz the continuous layer coordinate of a height z:
      0-2  p / 500 m          3  polar angle / pi     4  azimuth / pi
      5-7  e / 100 m          8  b_e(p) x 10          9  a(p) x 50
      10-12 d                 13 r / 100 m            14 c
      15 ln(1 + r / 1 m) / 5  16 2 delta              17 rho / 10 m
      18 exp(-|rho| / 2 m)    19 b_e(DOM) x 10        20 a(DOM) x 50
      21 mean b_e on the line x 10                    22 mean a on the line x 50
      23 r x mean a           24 r x mean b_e / 10
      25-27 exp(-r / 10, 30, 100 m)                   28 DOM z / 500 m
      29 e_z / max(r, 1 mm)   30 1 / (1 + r / 5 m)    31 r sin(acos c) / 100 m
    Point values use the layer containing the point (index clamped to the
    table); line means are path_mean over the heights of p and the DOM."""
    s = sources[np.asarray(pair_src)]
    cpos = np.asarray(dom_xyz, np.float64)[np.asarray(pair_dom)]
    d = np.stack([s["dx"], s["dy"], s["dz"]], 1).astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = np.stack([s["x"], s["y"], s["z"]], 1).astype(np.float64) + \
        0.5 * s["length"].astype(np.float64)[:, None] * d
    e = cpos - p
    r = np.linalg.norm(e, axis=1)
    rr = np.maximum(r, 1e-3)
    c = (d * e).sum(1) / rr
    th = np.arccos(np.clip(c, -1.0, 1.0))
    delta = th - theta_c
    rho = r * np.sin(delta)
    b_e = np.asarray(b_e, np.float64)
    a = np.asarray(a, np.float64)
    L = len(b_e)
    z_top = depth_of_z0 - depth_top
    us = (z_top - p[:, 2]) / dz
    ud = (z_top - cpos[:, 2]) / dz
    i_s, i_d = _layer_index(us, L), _layer_index(ud, L)
    mb, ma = path_mean(b_e, us, ud), path_mean(a, us, ud)
    f = np.zeros((len(s), IN))
    f[:, 0:3] = p / 500.0
    f[:, 3] = np.arccos(np.clip(d[:, 2], -1, 1)) / math.pi
    f[:, 4] = np.arctan2(d[:, 1], d[:, 0]) / math.pi
    f[:, 5:8] = e / 100.0
    f[:, 8] = b_e[i_s] * 10.0
    f[:, 9] = a[i_s] * 50.0
    f[:, 10:13] = d
    f[:, 13] = r / 100.0
    f[:, 14] = c
    f[:, 15] = np.log1p(r) / 5.0
    f[:, 16] = 2.0 * delta
    f[:, 17] = rho / 10.0
    f[:, 18] = np.exp(-np.abs(rho) / 2.0)
    f[:, 19] = b_e[i_d] * 10.0
    f[:, 20] = a[i_d] * 50.0
    f[:, 21] = mb * 10.0
    f[:, 22] = ma * 50.0
    f[:, 23] = r * ma
    f[:, 24] = r * mb / 10.0
    f[:, 25] = np.exp(-r / 10.0)
    f[:, 26] = np.exp(-r / 30.0)
    f[:, 27] = np.exp(-r / 100.0)
    f[:, 28] = cpos[:, 2] / 500.0
    f[:, 29] = e[:, 2] / rr
    f[:, 30] = 1.0 / (1.0 + r / 5.0)
    f[:, 31] = r * np.sqrt(np.maximum(0.0, 1.0 - c * c)) / 100.0
    return f


def _silu(z):
    return z / (1.0 + np.exp(-z))


def hswish(z):
    z = np.asarray(z, np.float64)
    return z * np.clip(z / 6.0 + 0.5, 0.0, 1.0)


def hswish_grad(z):
    z = np.asarray(z, np.float64)
    u = z / 6.0 + 0.5
    t = np.clip(u, 0.0, 1.0)
    return np.where((u > 0.0) & (u < 1.0), t + z / 6.0, t)


def _silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _softplus(z):
    return np.where(z > 20.0, z, np.log1p(np.exp(np.minimum(z, 20.0))))


def _act(act):
    if act == "silu":
        return _silu, _silu_grad
    if act == "hswish":
        return hswish, hswish_grad
    raise ValueError(act)


def forward(params, x, nph, rounding=True, act="silu"):
    """Returns lambda [n] and the cache the backward pass needs."""
    f, _ = _act(act)
    P = unpack(params)
    rnd = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    h = rnd(x)
    cache = {"x": h, "h": [], "z": []}
    for l in (1, 2, 3, 4):
        W = rnd(P[f"W{l}"])
        z = h @ W.T + P[f"b{l}"]
        cache["z"].append(rnd(z))
        h = rnd(f(z))
        cache["h"].append(h)
    zf = h @ P["w5"] + P["b5"]
    lam = np.asarray(nph, np.float64) * _softplus(zf)
    cache["zf"] = zf
    cache["lam"] = lam
    return lam, cache


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, "Adam: A Method for Stochastic
    Optimization", ICLR 2015, Algorithm 1), float64, elementwise.

    t is the number of the step being taken (1 for the first).  The moments
    are exponential moving averages of the gradient and of its square; the
    bias-corrected averages m_hat = m / (1 - b1^t), v_hat = v / (1 - b2^t)
    set the step -lr * m_hat / (sqrt(v_hat) + eps).  Returns (p, m, v) after
    the step; the inputs are not modified."""
    p, g, m, v = (np.asarray(a, np.float64) for a in (p, g, m, v))
    m_new = b1 * m + (1.0 - b1) * g
    v_new = b2 * v + (1.0 - b2) * g * g
    m_hat = m_new / (1.0 - b1 ** t)
    v_hat = v_new / (1.0 - b2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m_new, v_new


def loss_and_grads(params, x, nph, counts, rounding=True, act="silu"):
    """Mean Poisson NLL and its gradient with respect to every parameter."""
    _, fgrad = _act(act)
    P = unpack(params)
    rnd = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    lam, c = forward(params, x, nph, rounding, act)
    n = np.asarray(counts, np.float64)
    npairs = len(lam)
    lam_c = np.maximum(lam, 1e-300)
    loss = float(np.mean(lam_c - np.where(n > 0, n * np.log(lam_c), 0.0)))
    sig = 1.0 / (1.0 + np.exp(-c["zf"]))
    g = np.asarray(nph, np.float64) * sig * (1.0 - n / lam_c) / npairs   # dL/dz
    G = {"w5": c["h"][3].T @ g, "b5": g.sum()}
    dz = rnd(g[:, None] * P["w5"][None, :] * fgrad(c["z"][3]))
    for l in (4, 3, 2, 1):
        x_in = c["h"][l - 2] if l > 1 else c["x"]
        G[f"W{l}"] = dz.T @ x_in
        G[f"b{l}"] = dz.sum(0)
        if l > 1:
            W = rnd(P[f"W{l}"])
            dz = rnd((dz @ W) * fgrad(c["z"][l - 2]))
    return loss, pack(G)
