"""B300-native Monte Carlo photon propagation through layered ice.

The hot path is the CUDA library ``libpp.so`` (sources in ``csrc/``, C ABI in
``include/pp.h``); ``pp`` is its Python binding and ``workloads`` builds the
seeded synthetic inputs.  ``pp`` is imported on demand and raises if the
library has not been built -- nothing here computes on the CPU instead.
"""
__all__ = ["workloads", "pp"]
