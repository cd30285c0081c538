"""GB300-native electron-swarm Monte Carlo (null-collision step loop of
Betaboltz, arXiv:1901.08140) behind a C ABI.

Submodules are imported on demand: ``workloads`` (seeded synthetic inputs)
needs neither CUDA nor the compiled library; ``bz`` (the binding) loads the
CUDA library and fails loudly if it is missing.
"""
__all__ = ["workloads", "bz"]
