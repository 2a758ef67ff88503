"""GB300-native SDPD-DEM viscometer step (arXiv 2002.03120, "DEMocritus").

The compute path is the CUDA library ``libsdpd`` (``csrc/``) behind the C ABI
declared in ``include/sdpd.h``; ``binding`` is its thin ctypes wrapper and
``cases`` the seeded workload generators.  Importing the package does not load
the library; ``binding.load()`` does, and fails loudly if it is missing.
"""
__all__ = ["cases", "binding"]
