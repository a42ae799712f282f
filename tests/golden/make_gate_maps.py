"""Writes the oracle's per-DOM hit maps for the statistical parity gates
(oracle seeds 1001..1020; the GPU side runs seeds 1..20, so the two sides
draw independent streams).  Calls only the oracle and the input generators.

    python tests/golden/make_gate_maps.py [gate ...]

Gates (default: all):
  tiny_beside  tiny detector, an isotropic point source 3 m beside every DOM,
               1000 photons each (direct light on every DOM)
  tiny_point   the tiny-detector workload itself: one isotropic point source
               on the centre string at depth 1950 m, 2e7 photons per seed
               (diffuse light: tens of metres and ~60 scatters per photon)
  full_grid    the full-detector workload itself: the 1000 power-law
               muon-bundle events (41 degree Cherenkov segments), per-DOM hits
               summed over the events
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2405_05700_b300 import workloads as W  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
SEEDS = list(range(1001, 1021))
BESIDE_PHOTONS_PER_DOM = 1000
POINT_PHOTONS = 20_000_000


def gate_inputs(name):
    """(geometry, ice, batch, file name, extra npz fields) of a gate."""
    if name == "tiny_beside":
        return (W.geometry_tiny(), W.ice_tiny(), W.sources_gate(BESIDE_PHOTONS_PER_DOM),
                "gate_tiny_oracle.npz", {"photons_per_dom": BESIDE_PHOTONS_PER_DOM})
    if name == "tiny_point":
        return (W.geometry_tiny(), W.ice_tiny(), W.sources_tiny(POINT_PHOTONS),
                "gate_tiny_point_oracle.npz", {"photons": POINT_PHOTONS})
    if name == "full_grid":
        return (W.geometry_full(), W.ice_full(), W.events_full(), "gate_full_grid_oracle.npz",
                {"n_events": 1000})
    raise ValueError(name)


def make(name):
    geom, ice, batch, fname, extra = gate_inputs(name)
    maps, counts = [], []
    t0 = time.time()
    for s in SEEDS:
        h, c, _ = oracle.propagate(oracle.Model(geom, ice, seed=s), batch)
        maps.append(h.sum(0))
        counts.append(c.sum(0))
        print(f"{name} seed {s}: {int(h.sum())} hits, {time.time() - t0:.0f} s", flush=True)
    out = os.path.join(HERE, fname)
    np.savez_compressed(out, seeds=np.array(SEEDS), hits=np.array(maps, np.uint64),
                        counts=np.array(counts, np.uint64), **extra)
    print(f"wrote {out} in {time.time() - t0:.1f} s")


def main():
    names = sys.argv[1:] or ["tiny_beside", "tiny_point", "full_grid"]
    for n in names:
        make(n)


if __name__ == "__main__":
    main()
