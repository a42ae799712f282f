"""pp_propagate_noalloc: the entry point for callers that may not allocate
device memory during a call (it takes its scratch from a fixed static device
array instead of cudaMalloc-grown context buffers).

Checked through the C ABI against the allocating entry point pp_propagate on
the same events, on two calls in a row (the second call reuses the array the
first one left behind), for a warm call on a caller-owned stream that must
allocate nothing, and for the size limit.  The comparison is exact, as
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

        # a warm call on a caller-owned stream allocates nothing: the context's
        # device bytes and allocation count and the device's free memory are
        # unchanged across it; it launches its two kernels; its result and the
        # error check (pp_sync on that same stream) are ordered on that stream;
        # the caller's current device is left as it was
        e = events[-1]
        src = np.ascontiguousarray(batch.event(e))
        ev_id = int(batch.event_ids[e]) + 100
        want_h, want_c = prop.propagate(ev_id, src)
        d_src = torch.from_numpy(src.view(np.uint8).copy()).to(dev)
        d_hits = torch.full((geom.n_dom,), -1, dtype=torch.int64, device=dev)
        d_counts = torch.full((4,), -1, dtype=torch.int64, device=dev)
        user = torch.cuda.Stream()
        torch.cuda.synchronize()
        pp.pp_set_kernel_timing(prop.ctx, False)
        pp.pp_get_kernel_time(prop.ctx)                      # reset the launch count
        mem0 = pp.pp_get_memory(prop.ctx)
        free0 = torch.cuda.mem_get_info()[0]
        device0 = torch.cuda.current_device()
        pp.pp_propagate_noalloc(prop.ctx, ev_id, d_src, len(src), d_hits, d_counts,
                                user.cuda_stream)
        pp.pp_sync(prop.ctx, user.cuda_stream)
        assert torch.cuda.mem_get_info()[0] == free0
        assert pp.pp_get_memory(prop.ctx) == mem0
        assert pp.pp_get_kernel_time(prop.ctx)[2] == 2
        assert torch.cuda.current_device() == device0
        with torch.cuda.stream(user):
            got_h = d_hits.cpu().numpy().astype(np.uint64)
            got_c = d_counts.cpu().numpy().astype(np.uint64)
        assert np.array_equal(got_h, want_h) and np.array_equal(got_c, want_c)

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
