"""GB300-native X-drop seed-and-extend alignment.

The CUDA library (``libxdrop.so``, built from ``csrc/``) holds every step of
the alignment path; ``xdrop`` is its thin ctypes binding.  ``workloads``
draws seeded synthetic inputs.  Importing this package loads nothing; the
binding loads the library on first use and raises if it is missing.
"""
__all__ = ["xdrop", "workloads"]
