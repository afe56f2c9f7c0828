"""GB300-native isogeometric boundary element method for acoustic scattering (CFIE + FMM + GMRES).

The compute path is the CUDA library ``libigabem.so`` (C ABI in ``include/igabem.h``), loaded by
``binding``; ``inputs`` holds the seeded synthetic workloads.
"""
