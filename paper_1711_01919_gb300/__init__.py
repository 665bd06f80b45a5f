"""GB300-native integral histograms (arXiv 1711.01919).

The compute path is the CUDA library ``libihist.so`` built from ``csrc/``
(see ``include/ihist.h``); ``ihist`` is its thin ctypes binding.  ``synth``
holds the seeded input generators.
"""
__all__ = ["synth"]
