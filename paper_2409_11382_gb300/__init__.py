"""GB300-native (sm_103a) solver for Biot's consolidation model by the coupled
lattice Boltzmann method of Lunowa & Wohlmuth (arXiv 2409.11382).

The compute path is the C-ABI library ``libbiot_gb300.so`` (``include/biot.h``);
``biot.Solver`` is its thin Python binding and ``workloads`` builds the seeded
synthetic problems.  Importing the package does not load the library.
"""
__all__ = ["biot", "workloads", "build"]
