"""Oracle of the learned surrogate: the MLP's features, forward pass, loss and
gradients, written out plainly in numpy float64.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's checks); it does
not import the CUDA library.

The network (the surrogate has no counterpart in the paper; its definition is
the task's: BF16 weights, FP32 accumulation, Poisson mean output):
    h1 = silu(W1 x + b1), h_l = silu(W_l h_{l-1} + b_l) (l = 2..4),
    z = w5 . h4 + b5,  lambda = n_photons * softplus(z),
    loss = mean over pairs of (lambda - n ln lambda).
With rounding=True the values the device stores in BF16 are rounded to BF16
at the same points (weights W1..W4, inputs, hidden activations, the stored
pre-activations used by the backward pass, and the back-propagated dL/dz of
each layer); everything else is float64.  With rounding=False it is the plain
float64 network, which the finite-difference pin checks.
"""
from __future__ import annotations

import math

import numpy as np

HID, IN = 256, 16
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


def features(sources, pair_src, pair_dom, dom_xyz, b_e, a, depth_top, dz, depth_of_z0=1950.0):
    """The 16 inputs of each (source, DOM) pair, float64, unrounded:
    source point (segment midpoint) / 500 m, direction polar and azimuth angle
    / pi, DOM position relative to the point / 100 m, effective scattering x 10
    and absorption x 50 at the point's layer (depth rows clamped to the
    table), the unit direction, distance / 100 m, cosine between direction and
    the line to the DOM, ln(1 + distance / 1 m) / 5."""
    s = sources[np.asarray(pair_src)]
    c = np.asarray(dom_xyz, np.float64)[np.asarray(pair_dom)]
    d = np.stack([s["dx"], s["dy"], s["dz"]], 1).astype(np.float64)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = np.stack([s["x"], s["y"], s["z"]], 1).astype(np.float64) + \
        0.5 * s["length"].astype(np.float64)[:, None] * d
    e = c - p
    r = np.linalg.norm(e, axis=1)
    z_top = depth_of_z0 - depth_top
    li = np.clip(np.floor((z_top - p[:, 2]) / dz).astype(np.int64), 0, len(b_e) - 1)
    f = np.zeros((len(s), IN))
    f[:, 0:3] = p / 500.0
    f[:, 3] = np.arccos(np.clip(d[:, 2], -1, 1)) / math.pi
    f[:, 4] = np.arctan2(d[:, 1], d[:, 0]) / math.pi
    f[:, 5:8] = e / 100.0
    f[:, 8] = np.asarray(b_e, np.float64)[li] * 10.0
    f[:, 9] = np.asarray(a, np.float64)[li] * 50.0
    f[:, 10:13] = d
    f[:, 13] = r / 100.0
    f[:, 14] = (d * e).sum(1) / np.maximum(r, 1e-3)
    f[:, 15] = np.log1p(r) / 5.0
    return f


def _silu(z):
    return z / (1.0 + np.exp(-z))


def _silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def _softplus(z):
    return np.where(z > 20.0, z, np.log1p(np.exp(np.minimum(z, 20.0))))


def forward(params, x, nph, rounding=True):
    """Returns lambda [n] and the cache the backward pass needs."""
    P = unpack(params)
    rnd = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    h = rnd(x)
    cache = {"x": h, "h": [], "z": []}
    for l in (1, 2, 3, 4):
        W = rnd(P[f"W{l}"])
        z = h @ W.T + P[f"b{l}"]
        cache["z"].append(rnd(z))
        h = rnd(_silu(z))
        cache["h"].append(h)
    zf = h @ P["w5"] + P["b5"]
    lam = np.asarray(nph, np.float64) * _softplus(zf)
    cache["zf"] = zf
    cache["lam"] = lam
    return lam, cache


def loss_and_grads(params, x, nph, counts, rounding=True):
    """Mean Poisson NLL and its gradient with respect to every parameter."""
    P = unpack(params)
    rnd = bf16 if rounding else (lambda v: np.asarray(v, np.float64))
    lam, c = forward(params, x, nph, rounding)
    n = np.asarray(counts, np.float64)
    npairs = len(lam)
    lam_c = np.maximum(lam, 1e-300)
    loss = float(np.mean(lam_c - np.where(n > 0, n * np.log(lam_c), 0.0)))
    sig = 1.0 / (1.0 + np.exp(-c["zf"]))
    g = np.asarray(nph, np.float64) * sig * (1.0 - n / lam_c) / npairs   # dL/dz
    G = {"w5": c["h"][3].T @ g, "b5": g.sum()}
    dz = rnd(g[:, None] * P["w5"][None, :] * _silu_grad(c["z"][3]))
    for l in (4, 3, 2, 1):
        x_in = c["h"][l - 2] if l > 1 else c["x"]
        G[f"W{l}"] = dz.T @ x_in
        G[f"b{l}"] = dz.sum(0)
        if l > 1:
            W = rnd(P[f"W{l}"])
            dz = rnd((dz @ W) * _silu_grad(c["z"][l - 2]))
    return loss, pack(G)
