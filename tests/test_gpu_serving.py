"""The serving loop (pp_server): many host threads submit photon bunches, one
scheduler admits them under a budget and runs them in continuous batches.

* Each bunch's result in the concurrent mix equals its result alone (the
  plain single-event path), bit for bit, and conserves photons.
* Admission: a bunch costing more than the whole budget is refused; under a
  small budget every bunch still completes and the admitted total never
  exceeds the budget.
* pp_collect honours its timeout; unknown tickets and bad sources are refused;
  the context refuses new tables while a server is attached.
"""
import threading

import numpy as np
import pytest

from paper_2405_05700_b300 import workloads as W

pytestmark = pytest.mark.gpu


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


def test_results_in_the_mix_equal_results_alone(pp, prop):
    n_clients, per_client = 16, 6
    work = {c: _bunches(c, per_client) for c in range(n_clients)}
    got = {}
    errors = []
    with pp.Server(prop, slots=3) as server:
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
            rc, h, cnt = got[ev]
            assert rc == pp.PP_OK
            h1, c1 = prop.propagate(ev, src)
            assert np.array_equal(h, h1) and np.array_equal(cnt, c1), ev
            assert int(h.sum() + cnt[0] + cnt[1]) == int(src["n_photons"].sum())
    assert stats["bunches"] == n_clients * per_client
    assert stats["batches"] >= 1 and stats["p99_ms"] >= stats["p50_ms"] > 0


def test_admission_budget(pp, prop):
    bunches = _bunches(99, 20, pmax=2e5)
    costs = [int(s["n_photons"].sum()) * 32 + len(s) * 68 + 5160 * 8 + 64 for _, s in bunches]
    budget = 2 * max(costs)
    with pp.Server(prop, budget_bytes=budget, slots=3) as server:
        # a bunch alone above the budget is refused at once
        big = W.point_source(0.0, 0.0, 0.0, budget // 32 + 1)
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


def test_collect_timeout_unknown_ticket_and_bad_input(pp, prop):
    with pp.Server(prop, photon_state_bytes=1) as server:
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
        # the context keeps its tables while the server is attached
        geom = W.geometry_tiny()
        with pytest.raises(pp.PPError):
            pp.pp_load_geometry(prop.ctx, geom.xyz, geom.string_id, geom.n_dom, geom.dom_radius)
