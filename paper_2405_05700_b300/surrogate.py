"""Training and evaluation of the learned surrogate through the C ABI.

Host orchestration only: sources are drawn with numpy and moved with torch
(device buffers, index gathers); Monte Carlo runs in the propagation kernels,
the pair search, features, forward, backward and Adam in the surrogate's
kernels.

* make_training_set: sources propagated by Monte Carlo, one event per source;
  every (source, DOM) pair within r_max becomes a training pair with its hit
  count (pairs farther out carry no light worth learning: beyond 250 m the
  Monte Carlo light of the full detector is ~3e-4 of the total).
* train: Adam steps over shuffled batches, cosine learning-rate decay.
* evaluate: per-DOM expected hits of fresh sources from the surrogate against
  Monte Carlo hit counts (Pearson chi2 over DOMs expecting >= 5 hits), the
  time of each, and the hybrid that sends sources closer than r_fallback to a
  DOM to Monte Carlo.
"""
from __future__ import annotations

import dataclasses
import math
import time

import numpy as np

from . import pp, workloads as W


@dataclasses.dataclass
class TrainingSet:
    sources: np.ndarray
    feat: object         # torch int16 [P][32] (BF16 bits), on the device
    counts: object       # torch float32 [P]
    nph: object          # torch float32 [P]
    n_pairs: int
    mc_seconds: float


def _device_sources(src):
    import torch
    return torch.from_numpy(np.ascontiguousarray(src).view(np.uint8).copy()).cuda()


def mc_hits(prop, src, event_base, chunk=2000, event_ids=None):
    """Monte Carlo hits [n_src][n_dom] with one event per source (event ids
    event_base + i, or the given ones); returns (hits, seconds of device time)."""
    import torch
    stream = _stream(prop)
    ids = np.arange(event_base, event_base + len(src), dtype=np.int64) if event_ids is None \
        else np.asarray(event_ids, np.int64)
    with torch.cuda.stream(stream):
        return _mc_hits(prop, src, ids, chunk, stream)


def _mc_hits(prop, src, event_ids, chunk, stream):
    import torch
    n, n_dom = len(src), prop.n_dom
    out = np.zeros((n, n_dom), np.int64)
    secs = 0.0
    for c0 in range(0, n, chunk):
        part = np.ascontiguousarray(src[c0:c0 + chunk])
        m = len(part)
        d_src = _device_sources(part)
        ids = torch.from_numpy(event_ids[c0:c0 + m].copy()).cuda()
        beg = torch.arange(0, m + 1, dtype=torch.int64, device="cuda")
        hits = torch.zeros((m, n_dom), dtype=torch.int64, device="cuda")
        cnt = torch.zeros((m, 4), dtype=torch.int64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pp.pp_propagate_batch_async(prop.ctx, m, ids, beg, d_src, m, hits, cnt,
                                    stream.cuda_stream)
        e1.record(stream)
        pp.pp_sync(prop.ctx, stream.cuda_stream)
        secs += e0.elapsed_time(e1) * 1e-3
        out[c0:c0 + m] = hits.cpu().numpy()
    return out, secs


def _stream(prop):
    """The torch view of the context's CUDA stream: torch ops of this module
    run on it, so they are ordered with the library's work (the Propagator
    must have been created with an explicit stream)."""
    import torch
    if not prop.stream:
        raise ValueError("create the Propagator with stream=<a CUDA stream handle>")
    return torch.cuda.ExternalStream(prop.stream)


def make_training_set(prop, mlp, n_sources, photons, r_max=250.0, seed=0, event_base=0,
                      near_fraction=0.0, r_near=25.0):
    """Training pairs from n_sources Monte Carlo sources: a fraction
    near_fraction of them placed within r_near of a DOM, the rest uniform in
    the instrumented volume."""
    import torch
    with torch.cuda.stream(_stream(prop)):
        return _make_training_set(prop, mlp, n_sources, photons, r_max, seed, event_base,
                                  near_fraction, r_near)


def _near_pairs(mlp, d_src, n_src, r_max):
    """Device lists (pair_src, pair_dom) of the pairs closer than r_max."""
    import torch
    n = pp.pp_mlp_near_pairs(mlp.handle, d_src, n_src, r_max, 0, None, None)
    ps = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    pd = torch.zeros(max(n, 1), dtype=torch.int32, device="cuda")
    got = pp.pp_mlp_near_pairs(mlp.handle, d_src, n_src, r_max, n, ps, pd)
    assert got == n
    return ps[:n], pd[:n]


def _make_training_set(prop, mlp, n_sources, photons, r_max, seed, event_base, near_fraction,
                       r_near, chunk=2000):
    import torch
    rng = np.random.default_rng(seed)
    n_near = int(round(near_fraction * n_sources))
    parts = [W.surrogate_sources(rng, n_sources - n_near, photons)]
    if n_near:
        parts.append(W.surrogate_sources_near(rng, n_near, photons, prop.geom_xyz, r_near))
    src = np.concatenate(parts)
    d_src = _device_sources(src)
    stream = _stream(prop)
    all_ps, all_pd, all_cn = [], [], []
    secs = 0.0
    rec = src.dtype.itemsize
    for c0 in range(0, n_sources, chunk):
        m = min(chunk, n_sources - c0)
        part = d_src[c0 * rec:(c0 + m) * rec]
        # Monte Carlo counts of the chunk, one event per source, kept on the device
        ids = torch.arange(event_base + c0, event_base + c0 + m, dtype=torch.int64, device="cuda")
        beg = torch.arange(0, m + 1, dtype=torch.int64, device="cuda")
        hits = torch.zeros((m, prop.n_dom), dtype=torch.int64, device="cuda")
        cnt = torch.zeros((m, 4), dtype=torch.int64, device="cuda")
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pp.pp_propagate_batch_async(prop.ctx, m, ids, beg, part, m, hits, cnt, stream.cuda_stream)
        e1.record(stream)
        pp.pp_sync(prop.ctx, stream.cuda_stream)
        secs += e0.elapsed_time(e1) * 1e-3
        # the chunk's pairs within r_max and their counts
        ps, pd = _near_pairs(mlp, part, m, r_max)
        all_cn.append(hits[ps.long(), pd.long()].to(torch.float32))
        all_ps.append(ps + c0)
        all_pd.append(pd)
    ps, pd, cn = torch.cat(all_ps), torch.cat(all_pd), torch.cat(all_cn)
    n_pairs = int(ps.numel())
    feat = torch.zeros((n_pairs, pp.PP_MLP_INPUTS), dtype=torch.int16, device="cuda")
    pp.pp_mlp_features(mlp.handle, d_src, ps, pd, n_pairs, feat)
    pp.pp_mlp_sync(mlp.handle)
    nph = torch.full((n_pairs,), float(photons), dtype=torch.float32, device="cuda")
    return TrainingSet(src, feat, cn, nph, n_pairs, secs)


def train(mlp, data, epochs, batch=16384, lr=1e-3, lr_final_frac=0.03, seed=0, max_steps=None):
    """Adam over shuffled batches; returns the mean loss of each epoch."""
    import torch
    with torch.cuda.stream(_stream(mlp.prop)):
        return _train(mlp, data, epochs, batch, lr, lr_final_frac, seed, max_steps)


def _train(mlp, data, epochs, batch, lr, lr_final_frac, seed, max_steps):
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    steps_per_epoch = data.n_pairs // batch
    total = steps_per_epoch * epochs if max_steps is None else min(max_steps, steps_per_epoch * epochs)
    losses, k = [], 0
    for _ in range(epochs):
        perm = torch.randperm(data.n_pairs, device="cuda", generator=g)
        pp.pp_mlp_loss(mlp.handle)
        done = 0
        for i in range(steps_per_epoch):
            if k >= total:
                break
            rows = perm[i * batch:(i + 1) * batch]
            rate = lr * (lr_final_frac + (1 - lr_final_frac) * 0.5 * (1 + math.cos(math.pi * k / max(1, total))))
            pp.pp_mlp_train_step_rows(mlp.handle, data.feat, data.nph, data.counts, data.n_pairs,
                                      rows, batch, rate)
            k += 1
            done += 1
        losses.append(pp.pp_mlp_loss(mlp.handle) / max(1, done))
        if k >= total:
            break
    return losses


def evaluate(prop, mlp, n_sources, photons, seed=123, event_base=10_000_000,
             r_fallbacks=(0.0, 3.0, 5.0, 10.0), min_expected=5.0, r_max=250.0):
    """Surrogate vs Monte Carlo on fresh sources, per-DOM sums over sources.

    Surrogate alone: its per-DOM expectation against one MC run (Pearson
    chi2 / ndf over DOMs expecting >= min_expected hits).  Hybrid, for each
    fallback radius: sources closer than the radius to a DOM go to MC (the
    same events, hence the same counts), the rest to the surrogate, each part
    timed on its own; compared with an independent MC run of all sources
    (variance: the surrogate part's expectation + twice the MC part's
    counts).  Speedup = full MC time / surrogate (+ fallback MC) time."""
    import torch
    with torch.cuda.stream(_stream(prop)):
        return _evaluate(prop, mlp, n_sources, photons, seed, event_base, r_fallbacks,
                         min_expected, r_max)


def _sur_time(prop, mlp, src, photons, r_max, lam_out=None):
    """(per-DOM sums, device seconds) of the surrogate over the sources."""
    import torch
    st = _stream(prop)
    n = len(src)
    sums = torch.zeros(prop.n_dom, dtype=torch.float64, device="cuda")
    if n == 0:
        return sums.cpu().numpy(), 0.0
    d_src = _device_sources(src)
    nph = torch.full((n,), float(photons), dtype=torch.float32, device="cuda")
    pp.pp_mlp_dom_sums(mlp.handle, d_src, n, nph, r_max, sums, lam_out, st.cuda_stream)  # warm
    st.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    pp.pp_mlp_dom_sums(mlp.handle, d_src, n, nph, r_max, sums, None, st.cuda_stream)
    e1.record(st)
    st.synchronize()
    pp.pp_mlp_sync(mlp.handle)
    return sums.cpu().numpy(), e0.elapsed_time(e1) * 1e-3


def _evaluate(prop, mlp, n_sources, photons, seed, event_base, r_fallbacks, min_expected, r_max):
    import torch
    src = W.surrogate_sources(np.random.default_rng(seed), n_sources, photons)
    ids = np.arange(event_base, event_base + n_sources, dtype=np.int64)
    hits, mc_secs = mc_hits(prop, src, 0, event_ids=ids)
    hits2, _ = mc_hits(prop, src, 0, event_ids=ids + 5_000_000)   # independent reference run
    ref = hits2.sum(0).astype(np.float64)
    lam = torch.zeros((n_sources, prop.n_dom), dtype=torch.float32, device="cuda")
    sur_dom, sur_secs = _sur_time(prop, mlp, src, photons, r_max, lam)
    lam = lam.cpu().numpy().astype(np.float64)

    def chi2(resid2, var):
        use = var >= min_expected
        return float((resid2[use] / var[use]).sum()) / max(1, int(use.sum())), int(use.sum())

    res = {"sources": n_sources, "photons_per_source": photons, "mc_seconds": mc_secs,
           "surrogate_seconds": sur_secs, "speedup": mc_secs / sur_secs if sur_secs > 0 else None}
    res["chi2_ndf"], res["ndf"] = chi2((hits.sum(0) - sur_dom) ** 2, sur_dom)
    # per (source, DOM) pair, where errors of opposite sign cannot cancel as
    # they can in per-DOM sums: Pearson chi2 over pairs expecting >= min_expected
    # hits, the Poisson deviance per pair over every pair the surrogate
    # evaluates (expectation below 1 for pairs with few expected hits), and the
    # ratio of all MC hits to all expected hits
    n_pair = hits.astype(np.float64)
    use = lam >= min_expected
    modelled = lam > 0
    dev = 2.0 * (np.where(n_pair > 0, n_pair * np.log(np.maximum(n_pair, 1e-300) /
                                                     np.maximum(lam, 1e-300)), 0.0)
                 - (n_pair - lam))
    res["per_pair"] = {
        "chi2_ndf": float(((n_pair - lam) ** 2 / np.where(use, lam, 1.0))[use].sum())
                    / max(1, int(use.sum())),
        "ndf": int(use.sum()), "min_expected": min_expected,
        "deviance_per_pair": float(dev[modelled].sum()) / max(1, int(modelled.sum())),
        "pairs": int(modelled.sum()),
        "hits_over_expected": float(n_pair[modelled].sum() / max(lam[modelled].sum(), 1e-300))}
    # MC time grows with the photons per source, the surrogate's does not:
    # the speedup at a tenth of the photons as well
    src10 = src.copy()
    src10["n_photons"] = max(1, photons // 10)
    _, mc10 = mc_hits(prop, src10, 0, event_ids=ids + 7_000_000)
    res["speedup_by_photons"] = [
        {"photons_per_source": photons, "mc_seconds": mc_secs,
         "speedup": mc_secs / sur_secs if sur_secs > 0 else None},
        {"photons_per_source": int(src10["n_photons"][0]), "mc_seconds": mc10,
         "speedup": mc10 / sur_secs if sur_secs > 0 else None}]
    d_src = _device_sources(src)
    res["hybrid"] = []
    for r_fb in r_fallbacks:
        fb = np.zeros(n_sources, bool)
        if r_fb > 0:
            near_src, _ = _near_pairs(mlp, d_src, n_sources, r_fb)
            fb[near_src.cpu().numpy()] = True
        pred = lam[~fb].sum(0) + hits[fb].sum(0)
        var = lam[~fb].sum(0) + 2.0 * hits[fb].sum(0)
        c2, ndf = chi2((pred - ref) ** 2, var)
        _, t_sur = _sur_time(prop, mlp, src[~fb], photons, r_max)
        t_mc = mc_hits(prop, src[fb], 0, event_ids=ids[fb])[1] if fb.any() else 0.0
        t = t_sur + t_mc
        res["hybrid"].append({"r_fallback": r_fb, "fallback_fraction": float(fb.mean()),
                              "chi2_ndf": c2, "ndf": ndf, "seconds": t,
                              "speedup": mc_secs / t if t > 0 else None})
    return res
