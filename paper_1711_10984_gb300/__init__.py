"""GB300-native coupled lattice-Boltzmann / finite-difference solver for
chemically self-propelled droplets (Fadda, Gonnella, Lamura & Tiribocchi,
arXiv 1711.10984).

The compute path is the CUDA library ``liblbd.so`` (C ABI in ``include/lbd.h``);
``lbd`` is its thin ctypes binding and ``inputs`` builds seeded initial fields.
Importing the package loads nothing; ``lbd.load()`` loads the library and
raises if it has not been built.
"""
__all__ = ["lbd", "inputs"]
