"""The serving loop (pp_server): many host threads submit photon bunches into a
request ring in device memory; a persistent serving kernel pulls their photons
while new bunches keep arriving.

* Each bunch's result in the concurrent mix equals its result alone (the
  plain single-event path), bit for bit, and conserves photons.
* Bunches admitted while the kernel runs are taken by the running kernel (one
  launch serves them all); a ring smaller than the bunches in flight reuses
  its slots and arena ranges with exact results.
* Admission: a bunch occupying more device bytes than the whole budget (or
  more sources than the arena) is refused; under a small budget every bunch
  still completes and the admitted bytes never exceed the budget.
* pp_collect honours its timeout; unknown tickets and bad sources are refused;
  a bunch without photons is complete at once; the context refuses new tables
  while a server is attached.
* A large bunch after a run of small ones gets the whole serving kernel.
"""
import threading
import time

import numpy as np
import pytest

from paper_2405_05700_b300 import workloads as W

pytestmark = pytest.mark.gpu

N_DOM = 5160


@pytest.fixture(scope="module")
def pp():
    from paper_2405_05700_b300 import build
    build.build()
    from paper_2405_05700_b300 import pp as mod
    return mod


@pytest.fixture(scope="module")
def prop(pp):
    p = pp.Propagator(W.geometry_full(), W.ice_full(), seed=5)
    yield p
    p.close()


def _bunches(client, n, pmax=3e5):
    rng = np.random.default_rng(1000 + client)
    return [(client * 1000 + k, W.serving_bunch(rng, photons_min=1e4, photons_max=pmax))
            for k in range(n)]


def _bytes_bound(src):
    """Upper bound of the device bytes a bunch occupies while admitted: 40 B
    per source, its photon prefix (8 B per source + 8), its chunk table (at
    most n_src + 1 chunks, 4 B each + 4), its output slot (8 B per DOM + 32)
    and its 64-byte ring entry."""
    n = len(src)
    return 40 * n + 8 * (n + 1) + 4 * (n + 2) + 8 * (N_DOM + 4) + 64


def _check_alone(pp, prop, ev, src, res):
    rc, h, cnt = res
    assert rc == pp.PP_OK, rc
    h1, c1 = prop.propagate(ev, src)
    assert np.array_equal(h, h1) and np.array_equal(cnt, c1), ev
    assert int(h.sum() + cnt[0] + cnt[1]) == int(src["n_photons"].sum())


def test_results_in_the_mix_equal_results_alone(pp, prop):
    n_clients, per_client = 16, 6
    work = {c: _bunches(c, per_client) for c in range(n_clients)}
    got = {}
    errors = []
    with pp.Server(prop) as server:
        def client(c):
            try:
                tickets = []
                for ev, src in work[c]:
                    tickets.append((ev, server.submit(ev, src)))
                    if len(tickets) > 3:              # keep a few bunches in flight
                        ev0, t0 = tickets.pop(0)
                        got[ev0] = server.collect(t0, timeout_ms=60_000)
                for ev0, t0 in tickets:
                    got[ev0] = server.collect(t0, timeout_ms=60_000)
            except Exception as exc:  # surfaced below
                errors.append(exc)

        threads = [threading.Thread(target=client, args=(c,)) for c in range(n_clients)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        stats = server.stats()
    assert not errors, errors
    assert len(got) == n_clients * per_client
    for c in range(n_clients):
        for ev, src in work[c]:
            _check_alone(pp, prop, ev, src, got[ev])
    assert stats["bunches"] == n_clients * per_client
    assert stats["kernel_launches"] >= 1 and stats["p99_ms"] >= stats["p50_ms"] > 0
    assert 0 < stats["peak_admitted_bytes"] < stats["device_bytes"]


def test_bunches_arriving_while_the_kernel_runs_join_it(pp, prop):
    """A long bunch keeps the serving kernel busy; bunches submitted meanwhile
    are published into the ring and claimed by that same launch."""
    big = W.point_source(0.0, 0.0, 0.0, 200_000_000)
    small = _bunches(7, 12)
    with pp.Server(prop, max_launch_ms=5000) as server:
        t_big = server.submit(1, big)
        time.sleep(0.02)
        tickets = [(ev, s, server.submit(ev, s)) for ev, s in small]
        res_small = [(ev, s, server.collect(t, timeout_ms=60_000)) for ev, s, t in tickets]
        rc, h, c = server.collect(t_big, timeout_ms=60_000)
        st = server.stats()
    assert rc == pp.PP_OK and int(h.sum() + c[0] + c[1]) == 200_000_000
    for ev, s, res in res_small:
        _check_alone(pp, prop, ev, s, res)
    assert st["kernel_launches"] == 1, st


def test_small_ring_reuses_slots_and_arena_exactly(pp, prop):
    """Four ring slots and an arena of 2048 sources for 40 bunches: slots and
    arena ranges are reused many times over while the kernel runs."""
    bunches = _bunches(11, 40, pmax=1e5)
    assert max(len(s) for _, s in bunches) <= 2048
    with pp.Server(prop, ring_requests=4, arena_sources=2048) as server:
        tickets = [(ev, s, server.submit(ev, s)) for ev, s in bunches]
        res = [(ev, s, server.collect(t, timeout_ms=60_000)) for ev, s, t in tickets]
    for ev, s, r in res:
        _check_alone(pp, prop, ev, s, r)


def test_admission_budget(pp, prop):
    bunches = _bunches(99, 20, pmax=2e5)
    budget = 2 * max(_bytes_bound(s) for _, s in bunches)
    with pp.Server(prop, budget_bytes=budget, arena_sources=4096) as server:
        # a bunch alone above the budget, or above the arena, is refused at once
        big = np.concatenate([W.point_source(0.0, 0.0, 0.0, 1)] * (budget // 40 + 1))
        with pytest.raises(pp.PPError) as ei:
            server.submit(1, big)
        assert ei.value.code == pp.PP_EBUDGET
        tickets = [(ev, s, server.submit(ev, s)) for ev, s in bunches]
        for ev, s, t in tickets:
            rc, h, c = server.collect(t, timeout_ms=60_000)
            assert rc == pp.PP_OK
            assert int(h.sum() + c[0] + c[1]) == int(s["n_photons"].sum())
        st = server.stats()
    assert 0 < st["peak_admitted_bytes"] <= budget
    assert st["bunches"] == len(bunches)
    with pp.Server(prop, arena_sources=100) as server:
        many = np.concatenate([W.point_source(0.0, 0.0, 0.0, 1)] * 101)
        with pytest.raises(pp.PPError) as ei:
            server.submit(2, many)
        assert ei.value.code == pp.PP_EBUDGET


def test_collect_timeout_unknown_ticket_and_bad_input(pp, prop):
    with pp.Server(prop) as server:
        t = server.submit(7, W.point_source(0.0, 0.0, 0.0, 300_000_000))
        rc, _, _ = server.collect(t, timeout_ms=1)
        assert rc == pp.PP_ETIMEDOUT                 # still running; the ticket stays valid
        rc, h, c = server.collect(t, timeout_ms=120_000)
        assert rc == pp.PP_OK and int(h.sum() + c[0] + c[1]) == 300_000_000
        rc, _, _ = server.collect(t, timeout_ms=0)   # released after a successful collect
        assert rc == pp.PP_EINVAL
        bad = W.point_source(np.inf, 0.0, 0.0, 10)
        with pytest.raises(pp.PPError) as ei:
            server.submit(8, bad)
        assert ei.value.code == pp.PP_EINVAL
        # no photons: complete at once, all zeros
        t0 = server.submit(9, W.point_source(0.0, 0.0, 0.0, 0))
        rc, h, c = server.collect(t0, timeout_ms=0)
        assert rc == pp.PP_OK and h.sum() == 0 and c.sum() == 0
        # the context keeps its tables while the server is attached
        geom = W.geometry_tiny()
        with pytest.raises(pp.PPError):
            pp.pp_load_geometry(prop.ctx, geom.xyz, geom.string_id, geom.n_dom, geom.dom_radius)
    # config checks: the ring size must be a power of two
    with pytest.raises(pp.PPError):
        pp.Server(prop, ring_requests=6)


def test_a_large_bunch_after_small_ones_gets_the_whole_kernel(pp, prop):
    """Small bunches one at a time leave most warps idle between them; a
    large bunch that follows must still run on the whole serving kernel (a
    launch ends as a whole, never warp by warp).  2e6 photons of the tiny
    point-source kind take ~5 ms on the whole kernel; on the few warps a
    warp-by-warp exit used to leave, up to the 200 ms launch limit."""
    with pp.Server(prop) as server:
        for k in range(6):
            t = server.submit(100 + k, W.point_source(0.0, 0.0, 0.0, 10_000))
            assert server.collect(t, timeout_ms=60_000)[0] == pp.PP_OK
        src = W.point_source(0.0, 0.0, 0.0, 2_000_000)
        t0 = time.perf_counter()
        t = server.submit(200, src)
        rc, h, c = server.collect(t, timeout_ms=60_000)
        ms = (time.perf_counter() - t0) * 1e3
    assert rc == pp.PP_OK and int(h.sum() + c[0] + c[1]) == 2_000_000
    assert ms < 60.0, ms
