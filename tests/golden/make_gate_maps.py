"""Writes gate_tiny_oracle.npz: the oracle's per-DOM hit maps for the
statistical parity gate (tiny detector, a point source beside every DOM,
oracle seeds 1001..1020).  Calls only the oracle and the input generators.

    python tests/golden/make_gate_maps.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2405_05700_b300 import workloads as W  # noqa: E402

SEEDS = list(range(1001, 1021))
PHOTONS_PER_DOM = 1000


def main():
    geom, ice = W.geometry_tiny(), W.ice_tiny()
    batch = W.sources_gate(PHOTONS_PER_DOM)
    maps, counts = [], []
    t0 = time.time()
    for s in SEEDS:
        h, c, _ = oracle.propagate(oracle.Model(geom, ice, seed=s), batch)
        maps.append(h[0])
        counts.append(c[0])
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "gate_tiny_oracle.npz")
    np.savez_compressed(out, seeds=np.array(SEEDS), hits=np.array(maps, np.uint64),
                        counts=np.array(counts, np.uint64),
                        photons_per_dom=PHOTONS_PER_DOM)
    print(f"wrote {out} in {time.time() - t0:.1f} s")


if __name__ == "__main__":
    main()
