"""pp_propagate_noalloc: the entry point for callers that may not allocate
device memory during a call (it takes its scratch from a fixed static device
array instead of cudaMalloc-grown context buffers).

Checked through the C ABI against the allocating entry point pp_propagate on
the same events, on two calls in a row (the second call reuses the array the
first one left behind), and for the size limit.  The comparison is exact, as
in the other tally tests: both paths draw the same Philox streams and count
with integer atomics.  Kept in a file of its own, collected last.
"""
import numpy as np
import pytest

from paper_2405_05700_b300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point_twice_in_a_row():
    import torch
    from paper_2405_05700_b300 import build
    build.build()
    from paper_2405_05700_b300 import pp

    geom, ice = W.geometry_full(), W.ice_full()
    batch = W.events_full(n_events=6, seed=41)
    sizes = batch.src_begin[1:] - batch.src_begin[:-1]
    events = [int(e) for e in np.argsort(sizes)[-2:]]       # two largest events
    assert all(0 < sizes[e] <= pp.PP_NOALLOC_MAX_SOURCES for e in events)
    dev = torch.device("cuda", 0)
    with pp.Propagator(geom, ice, seed=3) as prop:
        for call, e in enumerate(events):
            src = np.ascontiguousarray(batch.event(e))
            ev_id = int(batch.event_ids[e]) + 100 * call
            want_h, want_c = prop.propagate(ev_id, src)
            d_src = torch.from_numpy(src.view(np.uint8).copy()).to(dev)
            d_hits = torch.full((geom.n_dom,), -1, dtype=torch.int64, device=dev)
            d_counts = torch.full((4,), -1, dtype=torch.int64, device=dev)
            torch.cuda.synchronize()   # torch's fills are on its stream, the call on the context's
            pp.pp_propagate_noalloc(prop.ctx, ev_id, d_src, len(src), d_hits, d_counts)
            pp.pp_sync(prop.ctx)
            got_h = d_hits.cpu().numpy().astype(np.uint64)
            got_c = d_counts.cpu().numpy().astype(np.uint64)
            assert np.array_equal(got_h, want_h), call
            assert np.array_equal(got_c, want_c), call
            assert int(got_h.sum() + got_c[0] + got_c[1]) == int(src["n_photons"].sum())

        # more sources than the static array holds: refused, nothing enqueued
        big = np.ascontiguousarray(np.concatenate([batch.sources, batch.sources]))
        assert len(big) > pp.PP_NOALLOC_MAX_SOURCES
        d_big = torch.from_numpy(big.view(np.uint8).copy()).to(dev)
        d_hits = torch.zeros((geom.n_dom,), dtype=torch.int64, device=dev)
        d_counts = torch.zeros((4,), dtype=torch.int64, device=dev)
        with pytest.raises(pp.PPError) as ei:
            pp.pp_propagate_noalloc(prop.ctx, 1, d_big, len(big), d_hits, d_counts)
        assert ei.value.code == pp.PP_EINVAL
        assert "8192" in str(ei.value)
