"""GB300 (sm_103a) free-energy lattice Boltzmann library: CUDA kernels behind
a C ABI (include/lb.h) with a thin ctypes binding (``lb``).

Submodules are imported on demand so that ``inputs`` (seeded synthetic
workloads) and ``build`` load without the compiled library.
"""
