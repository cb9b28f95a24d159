"""GB300-native SPH time-step hot path (arXiv 1809.08013, Algorithm 1).

The compute path is the CUDA library ``libsph`` (sources under ``csrc/``,
C ABI in ``include/sph.h``); ``binding`` is its thin ctypes binding and
``ics`` the seeded input generators. Importing the package loads nothing;
``binding.load()`` loads (and if needed builds) the library and raises if it
cannot.
"""
__all__ = ["ics", "binding"]
