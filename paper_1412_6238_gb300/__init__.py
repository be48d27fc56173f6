"""GB300-native CSF lattice Boltzmann step for thermocapillary flow.

The compute path is the C-ABI library ``liblbe.so`` built from ``csrc/`` (CUDA
for sm_103a); ``lbe`` is its ctypes binding.  ``workloads`` builds seeded
synthetic inputs.  Importing the package does not load the library; the
binding loads it on first use and raises if it is missing.
"""
__all__ = ["workloads", "lbe"]
