"""Pins of the oracle's random numbers (CPU only).

Philox4x32-10 (Salmon et al., SC'11) is checked bit for bit against an
independent implementation, PyTorch's CPU engine header, on random counters and
keys; the uniform mapping is checked against its definition's properties
(odd multiples of 2^-24 inside (0, 1)) and for uniformity and lag correlation.
"""
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _aten_ref_binary(tmp_path_factory):
    import torch
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("PyTorch CPU Philox header not available")
    out = str(tmp_path_factory.mktemp("aten") / "philox_ref")
    subprocess.check_call(["g++", "-std=c++17", "-O1", "-I" + inc,
                           os.path.join(HERE, "philox_aten_ref.cpp"), "-o", out])
    return out


def test_philox_matches_independent_implementation(orc, tmp_path_factory):
    exe = _aten_ref_binary(tmp_path_factory)
    rng = np.random.default_rng(1234)
    n = 20000
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2 ** 32, size=(n, 2), dtype=np.uint64).astype(np.uint32)
    # structured corner cases: zero counter/key, all-ones, photon-style counters
    ctr[:4] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [7, 0, 1, 0], [123456, 1, 99999, 0]]
    key[:4] = [[0, 0], [0xFFFFFFFF] * 2, [0, 5], [42, 77]]
    text = "\n".join(" ".join(str(int(v)) for v in np.concatenate([c, k]))
                     for c, k in zip(ctr, key))
    res = subprocess.run([exe], input=text, capture_output=True, text=True, check=True)
    ref = np.array([[int(t) for t in line.split()] for line in res.stdout.strip().splitlines()],
                   dtype=np.uint64).astype(np.uint32)
    got = orc.philox(ctr, key)
    assert ref.shape == got.shape
    assert np.array_equal(ref, got)


def test_u01_definition(orc):
    x = np.array([0, 1, 255, 256, 0xFFFFFF00, 0xFFFFFFFF, 0x80000000], np.uint32)
    u = orc.u01(x)
    k = u * 2.0 ** 24
    assert np.all(k == np.round(k)) and np.all(np.round(k) % 2 == 1)
    assert u.min() == 2.0 ** -24 and u.max() == 1.0 - 2.0 ** -24
    # binary32 holds every value exactly
    assert np.all(u.astype(np.float32).astype(np.float64) == u)


def test_philox_uniformity_and_lag_correlation(orc):
    n = 1 << 18
    pid = np.arange(n, dtype=np.uint64)
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = pid.astype(np.uint32)
    ctr[:, 2] = 3  # a step block
    x = orc.philox(ctr, np.array([0, 7], np.uint32))
    # chi^2 on 2^16 bins of the top 16 bits, all four words pooled
    bins = np.bincount((x.ravel() >> 16).astype(np.int64), minlength=1 << 16)
    exp = x.size / (1 << 16)
    chi2 = float(((bins - exp) ** 2 / exp).sum())
    ndf = (1 << 16) - 1
    assert abs(chi2 - ndf) / np.sqrt(2 * ndf) < 5
    # adjacent photon ids (adjacent counters) are uncorrelated
    u = orc.u01(x[:, 0])
    r = np.corrcoef(u[:-1], u[1:])[0, 1]
    assert abs(r) * np.sqrt(n) < 4
    # words within one block are uncorrelated
    v = orc.u01(x[:, 1])
    r2 = np.corrcoef(u, v)[0, 1]
    assert abs(r2) * np.sqrt(n) < 4
