"""GB300-native HyperBall step (Boldi & Vigna, arXiv:1308.2144).

The compute path is the CUDA library built from ``csrc/`` (C ABI declared in
``include/hyperball.h``); ``hyperball`` is its thin ctypes binding and
``graphs`` builds seeded synthetic inputs.  Importing the package loads
nothing; the library is loaded on first use and a missing library is an
error, never a fallback.
"""
__all__ = ["hyperball", "graphs"]
